// Host planner: the paper's schedules (Alg. 1-3, the ad hoc rule, Alg. 6 with
// diagonalization), the QR pairing, and this library's pass planning (gate
// passes inside a tile, coset passes for Pauli strings).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "sv_internal.h"

namespace sv {
namespace {

inline int popc(uint64_t v) { return __builtin_popcountll(v); }
inline int hibit(uint64_t v) { return 63 - __builtin_clzll(v); }
inline int lobit(uint64_t v) { return __builtin_ctzll(v); }
inline uint64_t bit(int q) { return 1ull << q; }

int gate_nq(int kind) {
    switch (kind) {
    case SV_RY: case SV_RZ: case SV_MAT1: return 1;
    case SV_CZ: case SV_GIVENS: case SV_MAT2: return 2;
    case SV_DEXC: case SV_MAT4: return 4;
    default: return -1;
    }
}

uint64_t local_set(const std::vector<int32_t> &l2p, int nL) {
    uint64_t m = 0;
    for (size_t q = 0; q < l2p.size(); ++q)
        if (l2p[q] < nL) m |= bit((int)q);
    return m;
}

uint64_t to_physical(uint64_t logical, const std::vector<int32_t> &l2p) {
    uint64_t out = 0;
    while (logical) {
        int q = lobit(logical);
        logical &= logical - 1;
        out |= bit(l2p[q]);
    }
    return out;
}

// depth(U) = 0 if no earlier operator shares a qubit, else 1 + the largest
// depth among earlier operators sharing a qubit (critical path, Sec. III-A).
std::vector<int32_t> depths(const std::vector<Op> &ops) {
    int32_t last[64];
    std::fill(last, last + 64, -1);
    std::vector<int32_t> d(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        int32_t di = 0;
        for (int t = 0; t < ops[i].nq; ++t)
            if (last[ops[i].q[t]] >= 0) di = std::max(di, last[ops[i].q[t]] + 1);
        for (int t = 0; t < ops[i].nq; ++t) last[ops[i].q[t]] = di;
        d[i] = di;
    }
    return d;
}

// Ascending depth; ties by the sorted target tuple, then input position
// (Sec. IV-A-1).  The sort is stable, so equal keys keep input order.
std::vector<int32_t> depth_sort(const std::vector<Op> &ops) {
    std::vector<int32_t> d = depths(ops);
    std::vector<std::vector<int32_t>> key(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        key[i].assign(ops[i].q, ops[i].q + ops[i].nq);
        std::sort(key[i].begin(), key[i].end());
    }
    std::vector<int32_t> idx(ops.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        if (d[a] != d[b]) return d[a] < d[b];
        return key[a] < key[b];
    });
    return idx;
}

// Alg. 2 (P1): single scan in depth order.
void tile_construction(uint64_t QL, const std::vector<int32_t> &remain, const std::vector<Op> &ops,
                       std::vector<int32_t> &G) {
    uint64_t avail = QL;
    G.clear();
    for (int32_t u : remain) {
        uint64_t t = ops[u].tmask;
        if ((t & ~avail) == 0) G.push_back(u);
        else avail &= ~t;
        if (!avail) break;
    }
}

// Alg. 3 (P2), with the padding rule selectable.
uint64_t qubit_mapping(uint64_t Q, const std::vector<int32_t> &remain, const std::vector<Op> &ops,
                       int nL, bool pad_highest) {
    uint64_t avail = Q, QL = 0;
    for (int32_t u : remain) {
        uint64_t t = ops[u].tmask;
        if ((t & ~avail) == 0 && popc(QL | t) <= nL) QL |= t;
        else avail &= ~t;
        if (!avail) break;
    }
    if (!QL) return 0;
    uint64_t fr = Q & ~QL;
    while (popc(QL) < nL && fr) {
        int q = pad_highest ? hibit(fr) : lobit(fr);
        QL |= bit(q);
        fr &= ~bit(q);
    }
    return QL;
}

// Physical pairs of one QR: outgoing locals and incoming globals, each sorted
// by current physical position, swapped pairwise.  Updates l2p.
void qr_pairs(std::vector<int32_t> &l2p, uint64_t old_loc, uint64_t new_loc, std::vector<int32_t> &pairs) {
    std::vector<int32_t> out, in;
    for (uint64_t v = old_loc & ~new_loc; v; v &= v - 1) out.push_back(lobit(v));
    for (uint64_t v = new_loc & ~old_loc; v; v &= v - 1) in.push_back(lobit(v));
    auto bypos = [&](int32_t a, int32_t b) { return l2p[a] < l2p[b]; };
    std::sort(out.begin(), out.end(), bypos);
    std::sort(in.begin(), in.end(), bypos);
    pairs.clear();
    for (size_t i = 0; i < out.size() && i < in.size(); ++i) {
        int32_t pa = l2p[out[i]], pb = l2p[in[i]];
        pairs.push_back(pa);
        pairs.push_back(pb);
        l2p[out[i]] = pb;
        l2p[in[i]] = pa;
    }
}

bool is_diag_op(const Op &op) { return op.kind == SV_RZ || op.kind == SV_CZ; }

// Alg. 2 with diagonal gates exempt from locality: a diagonal gate is taken
// when no earlier skipped gate shares a qubit with it, whatever its targets.
void tile_construction_dx(uint64_t QL, const std::vector<int32_t> &remain, const std::vector<Op> &ops,
                          std::vector<int32_t> &G, uint64_t Q) {
    uint64_t blocked = 0;
    G.clear();
    for (int32_t u : remain) {
        const uint64_t t = ops[u].tmask;
        const bool ok = (t & blocked) == 0 && (is_diag_op(ops[u]) || (t & ~QL) == 0);
        if (ok) G.push_back(u);
        else blocked |= t;
        if ((blocked & Q) == Q) break;
    }
}

// Alg. 3 with diagonal gates exempt: they neither claim local qubits nor block.
uint64_t qubit_mapping_dx(uint64_t Q, const std::vector<int32_t> &remain, const std::vector<Op> &ops, int nL,
                          bool pad_highest) {
    std::vector<int32_t> nd;
    for (int32_t u : remain)
        if (!is_diag_op(ops[u])) nd.push_back(u);
    if (nd.empty()) return 0;
    return qubit_mapping(Q, nd, ops, nL, pad_highest);
}

std::string flat_tiling(int n, int nL, const std::vector<Op> &ops, bool pad_highest,
                        std::vector<int32_t> l2p, std::vector<int32_t> &order, std::vector<Tile> &tiles,
                        std::vector<int32_t> &final_l2p, bool dx) {
    const uint64_t Q = (n == 64) ? ~0ull : (bit(n) - 1);
    uint64_t cur = local_set(l2p, nL);
    uint64_t QL = cur;
    std::vector<int32_t> remain = depth_sort(ops), G, next;
    std::vector<char> taken(ops.size(), 0);
    int stall = 0;
    while (!remain.empty()) {
        if (dx) tile_construction_dx(QL, remain, ops, G, Q);
        else tile_construction(QL, remain, ops, G);
        if (!G.empty()) {
            Tile t;
            t.begin = (int32_t)order.size();
            order.insert(order.end(), G.begin(), G.end());
            t.end = (int32_t)order.size();
            t.local_mask = QL;
            if (QL != cur) qr_pairs(l2p, cur, QL, t.pairs);
            t.l2p = l2p;
            cur = QL;
            tiles.push_back(std::move(t));
            for (int32_t u : G) taken[u] = 1;
            next.clear();
            for (int32_t u : remain)
                if (!taken[u]) next.push_back(u);
            remain.swap(next);
            stall = 0;
        } else if (++stall > 1) {
            return "flat tiling made no progress";
        }
        if (remain.empty()) break;
        QL = dx ? qubit_mapping_dx(Q, remain, ops, nL, pad_highest) : qubit_mapping(Q, remain, ops, nL, pad_highest);
        if (!QL) return "qubit mapping returned an empty set";
    }
    final_l2p = l2p;
    return "";
}

// Alg. 4 with Alg. 5: flat tiling whose remapping first tries to draw the
// next local set from Q_L u Q_intra (an intra QR) and only otherwise selects
// the local and intra sets from all qubits (an inter QR).  Q_intra starts as
// the logical qubits at physical positions n_L .. n_L + n_intra - 1.
std::string hierarchical_tiling(int n, int nL, int nintra, const std::vector<Op> &ops, bool pad_highest,
                                std::vector<int32_t> l2p, std::vector<int32_t> &order, std::vector<Tile> &tiles,
                                std::vector<int32_t> &final_l2p) {
    const uint64_t Q = (n == 64) ? ~0ull : (bit(n) - 1);
    uint64_t cur = local_set(l2p, nL);
    uint64_t QL = cur, Qintra = 0;
    for (int q = 0; q < n; ++q)
        if (l2p[q] >= nL && l2p[q] < nL + nintra) Qintra |= bit(q);
    std::vector<int32_t> remain = depth_sort(ops), G, next;
    std::vector<char> taken(ops.size(), 0);
    int stall = 0;
    while (!remain.empty()) {
        tile_construction(QL, remain, ops, G);
        if (!G.empty()) {
            Tile t;
            t.begin = (int32_t)order.size();
            order.insert(order.end(), G.begin(), G.end());
            t.end = (int32_t)order.size();
            t.local_mask = QL;
            t.intra_mask = Qintra;
            if (QL != cur) qr_pairs(l2p, cur, QL, t.pairs);
            t.l2p = l2p;
            cur = QL;
            tiles.push_back(std::move(t));
            for (int32_t u : G) taken[u] = 1;
            next.clear();
            for (int32_t u : remain)
                if (!taken[u]) next.push_back(u);
            remain.swap(next);
            stall = 0;
        } else if (++stall > 1) {
            return "hierarchical tiling made no progress";
        }
        if (remain.empty()) break;
        const int nl = popc(QL), ni = popc(Qintra);
        uint64_t QLn = qubit_mapping(QL | Qintra, remain, ops, nl, pad_highest);
        if (QLn) {
            Qintra = (QL | Qintra) & ~QLn;
        } else {
            QLn = qubit_mapping(Q, remain, ops, nl, pad_highest);
            const uint64_t Qp = qubit_mapping(Q, remain, ops, nl + ni, pad_highest);
            Qintra = Qp & ~QLn;
        }
        QL = QLn;
        if (!QL) return "qubit mapping returned an empty set";
    }
    final_l2p = l2p;
    return "";
}

// The ad hoc rule: depth (or given) order; before an operation with a global
// target, evict as many locals outside its targets as it has global targets,
// least recently used first (never used = -1), ties to the highest index.
std::string adhoc_schedule(int n, int nL, const std::vector<Op> &ops, const std::vector<int32_t> &seq,
                           std::vector<int32_t> l2p, std::vector<int32_t> &order,
                           std::vector<Tile> &tiles, std::vector<int32_t> &final_l2p) {
    uint64_t QL = local_set(l2p, nL);
    std::vector<int64_t> last(n, -1);
    Tile cur;
    cur.begin = (int32_t)order.size();
    cur.local_mask = QL;
    cur.l2p = l2p;
    for (size_t x = 0; x < seq.size(); ++x) {
        int32_t u = seq[x];
        uint64_t t = ops[u].tmask;
        if (t & ~QL) {
            uint64_t inn = t & ~QL;
            int k = popc(inn);
            std::vector<int32_t> cand;
            for (uint64_t v = QL & ~t; v; v &= v - 1) cand.push_back(lobit(v));
            std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
                if (last[a] != last[b]) return last[a] < last[b];
                return a > b;
            });
            if ((int)cand.size() < k) return "operation wider than the local qubits";
            uint64_t evict = 0;
            for (int i = 0; i < k; ++i) evict |= bit(cand[i]);
            uint64_t newQL = (QL & ~evict) | inn;
            if ((int32_t)order.size() > cur.begin) {
                cur.end = (int32_t)order.size();
                tiles.push_back(cur);
            }
            cur = Tile();
            cur.begin = (int32_t)order.size();
            qr_pairs(l2p, QL, newQL, cur.pairs);
            QL = newQL;
            cur.local_mask = QL;
            cur.l2p = l2p;
        }
        order.push_back(u);
        for (int i = 0; i < ops[u].nq; ++i) last[ops[u].q[i]] = (int64_t)x;
    }
    if ((int32_t)order.size() > cur.begin) {
        cur.end = (int32_t)order.size();
        tiles.push_back(cur);
    }
    final_l2p = l2p;
    return "";
}

// ------------------------------------------------------------ gate passes --
// Inside a tile every gate is narrow.  Gates are grouped into passes that each
// stage 2^k amplitudes in shared memory: the staged physical set always holds
// the `low` lowest bits (coalesced runs) and is chosen like Alg. 3 (targets of
// the earliest remaining gates), padded with the lowest free local bits; the
// pass then takes gates like Alg. 2 (a gate that does not fit blocks its
// targets), which keeps the dependency order C1.
// Gates a pass staging S would take (the Alg. 2 scan: a gate that does not
// fit blocks its targets), at most cap.
int pass_take_count(const std::vector<int32_t> &remain, const std::vector<uint64_t> &pm, uint64_t S, int cap) {
    uint64_t av = S;
    int c = 0;
    for (int32_t u : remain) {
        const uint64_t t = pm[u];
        if ((t & ~av) == 0) {
            if (++c >= cap) break;
        } else {
            av &= ~t;
        }
        if (!av) break;
    }
    return c;
}

// Staged set of the next pass.  Two candidates: (a) the targets of the
// earliest remaining gates (Alg. 3 style), padded with the lowest free local
// bits; (b) grown from the low bits step by step, each step adding either one
// local bit or all missing targets of one of the earliest remaining gates,
// whichever lets the pass take the most gates per added bit (ties: fewer
// bits, then the earlier candidate).  (b) follows the light cone of a circuit
// instead of its earliest layer.  The candidate taking more gates wins, (a)
// on a tie.
uint64_t choose_staged(const std::vector<int32_t> &remain, const std::vector<uint64_t> &pm, uint64_t lowmask,
                       uint64_t localbits, int k, int cap) {
    uint64_t Sa = lowmask, avail = localbits;
    for (int32_t u : remain) {
        uint64_t t = pm[u];
        if ((t & ~avail) == 0 && popc(Sa | t) <= k) Sa |= t;
        else avail &= ~t;
        if (!avail || popc(Sa) == k) break;
    }
    for (uint64_t fr = localbits & ~Sa; popc(Sa) < k && fr; fr &= fr - 1) Sa |= bit(lobit(fr));
    // candidate bits in order of first appearance among the remaining targets
    std::vector<int> cand;
    uint64_t seen = lowmask;
    for (int32_t u : remain) {
        for (uint64_t t = pm[u] & localbits & ~seen; t; t &= t - 1) cand.push_back(lobit(t));
        seen |= pm[u] & localbits;
        if ((seen & localbits) == localbits) break;
    }
    uint64_t Sb = lowmask;
    const int base_c = pass_take_count(remain, pm, Sb, cap);
    int cur_c = base_c;
    while (popc(Sb) < k) {
        std::vector<uint64_t> adds;
        for (int b : cand)
            if (!(Sb >> b & 1)) adds.push_back(bit(b));
        int looked = 0;
        for (int32_t u : remain) {
            const uint64_t miss = pm[u] & localbits & ~Sb;
            if (popc(miss) > 1 && popc(Sb | miss) <= k) adds.push_back(miss);
            if (++looked >= 64) break;
        }
        uint64_t best = 0;
        double bestr = -1.0;
        int bestn = 0;
        for (uint64_t a : adds) {
            const int na = popc(a);
            const double r = (double)(pass_take_count(remain, pm, Sb | a, cap) - cur_c) / na;
            if (r > bestr || (r == bestr && na < bestn)) { bestr = r; best = a; bestn = na; }
        }
        if (!best) break;
        Sb |= best;
        cur_c = pass_take_count(remain, pm, Sb, cap);
    }
    for (uint64_t fr = localbits & ~Sb; popc(Sb) < k && fr; fr &= fr - 1) Sb |= bit(lobit(fr));
    return pass_take_count(remain, pm, Sb, cap) > pass_take_count(remain, pm, Sa, cap) ? Sb : Sa;
}

void plan_gate_passes(QsuPlan &P, const std::vector<Op> &ops, int k, int low, int fuse_max, bool dx) {
    const int nL = P.nL;
    const int cap = (fuse_max > 0 && fuse_max < kMaxPassOps) ? fuse_max : kMaxPassOps;
    k = std::min(k, nL);
    low = std::min(low, k);
    const uint64_t localbits = (nL == 64) ? ~0ull : (bit(nL) - 1);
    const uint64_t lowmask = bit(low) - 1;
    for (size_t ti = 0; ti < P.tiles.size(); ++ti) {
        const Tile &T = P.tiles[ti];
        std::vector<int32_t> remain(P.order.begin() + T.begin, P.order.begin() + T.end);
        std::vector<uint64_t> pm(ops.size(), 0);
        // under the diagonal exemption only the local targets of a gate are staged
        for (int32_t u : remain) pm[u] = to_physical(ops[u].tmask, T.l2p) & (dx ? localbits : ~0ull);
        std::vector<int32_t> G, next;
        while (!remain.empty()) {
            const uint64_t S = choose_staged(remain, pm, lowmask, localbits, k, cap);
            uint64_t av = S;
            G.clear();
            for (int32_t u : remain) {
                uint64_t t = pm[u];
                if ((t & ~av) == 0) G.push_back(u);
                else av &= ~t;
                if (!av || (int)G.size() >= cap) break;
            }
            GatePass gp;
            gp.tile = (int32_t)ti;
            gp.k = popc(S);
            int nl = 0;
            while (nl < 64 && (S >> nl & 1)) ++nl;
            gp.nlow = nl;
            gp.bits = S;
            gp.op_begin = (int32_t)P.ops.size();
            // tile-local position of each staged physical bit
            int8_t loc[64];
            int c = 0;
            for (int b = 0; b < 64; ++b)
                if (S >> b & 1) loc[b] = (int8_t)c++;
            for (int32_t u : G) {
                DevOp d;
                d.kind = ops[u].kind;
                for (int i = 0; i < 4; ++i) {
                    if (i >= ops[u].nq) { d.t[i] = -1; continue; }
                    const int pb = T.l2p[ops[u].q[i]];
                    d.t[i] = (int8_t)((S >> pb & 1) ? loc[pb] : kOutTarget + pb);
                }
                d.gate = u;
                d.mat = ops[u].mat;
                P.ops.push_back(d);
            }
            gp.op_end = (int32_t)P.ops.size();
            P.passes.push_back(gp);
            std::vector<char> in(ops.size(), 0);
            for (int32_t u : G) in[u] = 1;
            next.clear();
            for (int32_t u : remain)
                if (!in[u]) next.push_back(u);
            remain.swap(next);
        }
    }
}

// ------------------------------------------------------- register phases --
// A pass made only of RY, RZ, CZ and 1-qubit matrices is run register
// blocked: every thread holds 2^r amplitudes spanned by r tile bits (the
// register set).  Non-diagonal gates need their target in the register set;
// diagonal gates (RZ, CZ) apply in any layout.  Phases are built like the
// tiles: the register set takes the targets of the earliest remaining
// non-diagonal gates (padded with the lowest free tile bits), then the phase
// takes gates in order while they fit, a gate that does not fit blocking its
// targets (C1 is kept).  The pass's ops are reordered phase by phase.
bool diag_kind(int kind) { return kind == SV_RZ || kind == SV_CZ; }
int op_qubits(int kind) {
    return kind == SV_DEXC || kind == SV_MAT4 ? 4 : (kind == SV_CZ || kind == SV_GIVENS || kind == SV_MAT2) ? 2 : 1;
}

// Lane bits of a phase: the 5 tile bits outside the register set that the
// lane bits of the thread index hold.  A warp gathers its 32 x 2^r
// amplitudes by shared-memory slot swz_slot(base | v); for 8-byte (and
// 16-byte) elements it takes no extra bank wavefront when the lanes' slots
// differ in all 4 low bits, i.e. when the low-4-bit parts of the lane bits'
// slots have rank 4.  The lanes are picked greedily (lowest bits first) for
// that rank, then padded with the lowest remaining bits; the other thread
// index bits take the remaining bits in ascending order.
uint32_t phase_lanes(uint32_t rmask, int k) {
    uint32_t lanes = 0, span[4] = {0, 0, 0, 0};
    int rank = 0, nl = 0;
    for (int t = 0; t < k && nl < 5 && rank < 4; ++t) {
        if (rmask >> t & 1u) continue;
        uint32_t v = swz_slot(1u << t) & 15u;
        for (int i = 3; i >= 0; --i)
            if ((v >> i & 1u) && span[i]) v ^= span[i];
        if (!v) continue;
        span[31 - __builtin_clz(v)] = v;
        ++rank;
        lanes |= 1u << t;
        ++nl;
    }
    // the fifth lane bit (the half-warp bit) above the four independent ones,
    // so that lanes 0-15 of a warp hit 16 distinct slots mod 16
    const int top = lanes ? 31 - __builtin_clz(lanes) : -1;
    for (int t = top + 1; t < k && nl < 5; ++t)
        if (!(rmask >> t & 1u) && !(lanes >> t & 1u)) {
            lanes |= 1u << t;
            ++nl;
        }
    for (int t = 0; t < k && nl < 5; ++t)
        if (!(rmask >> t & 1u) && !(lanes >> t & 1u)) {
            lanes |= 1u << t;
            ++nl;
        }
    return lanes;
}

void plan_phases(QsuPlan &P, bool pairs) {
    for (auto &gp : P.passes) {
        const int r = gp.k - 9;                       // 512 threads
        if (r < 2) continue;
        bool ok = true;
        for (int o = gp.op_begin; o < gp.op_end; ++o) {
            const int kd = P.ops[o].kind;
            // a double excitation needs four register bits
            if (kd != SV_RY && kd != SV_RZ && kd != SV_CZ && kd != SV_MAT1 && !(pairs && kd == SV_GIVENS) &&
                !(pairs && kd == SV_DEXC && r == 4))
                ok = false;
        }
        if (!ok) continue;
        const uint32_t all = (gp.k >= 32) ? 0xFFFFFFFFu : ((1u << gp.k) - 1u);
        auto tmask = [&](const DevOp &d) {
            uint32_t m = 0;
            const int nq = op_qubits(d.kind);
            for (int i = 0; i < nq; ++i)
                if (d.t[i] < kOutTarget) m |= 1u << d.t[i];
            return m;
        };
        std::vector<DevOp> remain(P.ops.begin() + gp.op_begin, P.ops.begin() + gp.op_end), next, out;
        gp.ph_begin = (int32_t)P.phases.size();
        while (!remain.empty()) {
            uint32_t Rm = 0, avail = all;
            for (auto &d : remain) {
                const uint32_t t = tmask(d);
                if (diag_kind(d.kind)) {
                    if (t & ~avail) avail &= ~t;
                    continue;
                }
                if ((t & ~avail) == 0 && __builtin_popcount(Rm | t) <= r) Rm |= t;
                else avail &= ~t;
                if (!avail || __builtin_popcount(Rm) == r) break;
            }
            for (uint32_t fr = all & ~Rm; __builtin_popcount(Rm) < r && fr; fr &= fr - 1) Rm |= fr & (0u - fr);
            Phase ph;
            ph.rmask = Rm;
            ph.lanes = phase_lanes(Rm, gp.k);
            ph.st_begin = ph.st_end = 0;
            ph.op_begin = gp.op_begin + (int32_t)out.size();
            uint32_t av = all;
            next.clear();
            for (auto &d : remain) {
                const uint32_t t = tmask(d);
                const bool fits = (t & ~av) == 0 && (diag_kind(d.kind) || (t & ~Rm) == 0);
                if (fits) out.push_back(d);
                else {
                    av &= ~t;
                    next.push_back(d);
                }
            }
            ph.op_end = gp.op_begin + (int32_t)out.size();
            P.phases.push_back(ph);
            remain.swap(next);
        }
        gp.ph_end = (int32_t)P.phases.size();
        std::copy(out.begin(), out.end(), P.ops.begin() + gp.op_begin);
    }
}

// Steps of the register phases.  Inside a phase two operations on disjoint
// tile bits commute, and so do two diagonal operations (RZ, CZ) on any bits;
// every topological order of the "does not commute" relation applies the
// same operator.  Diagonal gates on thread bits only (no register bit) commute
// with every operation of the phase: they form one thread block at the
// phase's end.  The rest is rescheduled as a list of steps: all ready RY
// gates (distinct register bits) form one ROT step; when none is ready, other
// non-diagonal operations go one by one; when only diagonal ones are ready,
// all of them form one run, so that diagonal gates are delayed as long as
// possible and gather into few runs.  A run worth it becomes a register
// block, else its operations go one by one.  Blocks are made while the
// pass's shared memory allows.  In the adjoint sweep every RZ of a block
// takes its generator expectation at the block's end (Z commutes with the
// block), every RY of a ROT step at the step's end, and every RZ of a thread
// block anywhere in the phase (it commutes with the whole phase).
bool in_tile_diag(const DevOp &d) {
    return diag_kind(d.kind) && d.t[0] < kOutTarget && (d.kind != SV_CZ || d.t[1] < kOutTarget);
}

// A run is worth a register block when its members one by one cost more
// than one table lookup and complex product per amplitude: RZ ~ one complex
// product per amplitude, CZ ~ a quarter.
bool diag_run_pays(const std::vector<DevOp> &run) {
    int rz = 0, cz = 0;
    for (auto &d : run) (d.kind == SV_RZ ? rz : cz)++;
    return 4 * rz + cz >= 6;
}

void plan_steps(QsuPlan &P, int max_diag, int amp) {
    auto tm = [](const DevOp &d) {
        uint32_t m = 0;
        const int nq = op_qubits(d.kind);
        for (int i = 0; i < nq; ++i)
            if (d.t[i] >= 0 && d.t[i] < kOutTarget) m |= 1u << d.t[i];
        return m;
    };
    for (auto &gp : P.passes) {
        gp.db_begin = gp.db_end = (int32_t)P.dblocks.size();
        if (gp.ph_begin < 0) continue;
        const int nops = gp.op_end - gp.op_begin;
        int budget = kRegSmemLimit - reg_pass_fixed_bytes(gp.k, gp.nlow, nops, nops, gp.ph_end - gp.ph_begin, amp);
        int area = 0;   // bytes of the pass's block area handed out so far
        auto take_block = [&](int kind) {
            const int need = diag_block_bytes(kind, gp.k, amp);
            if ((int)P.dblocks.size() - gp.db_begin >= max_diag || need > budget) return -1;
            budget -= need;
            const int off = area;
            area += need;
            return off;
        };
        for (int ph = gp.ph_begin; ph < gp.ph_end; ++ph) {
            Phase &F = P.phases[ph];
            F.st_begin = (int32_t)P.steps.size();
            const std::vector<DevOp> all(P.ops.begin() + F.op_begin, P.ops.begin() + F.op_end);
            // thread-only diagonal operations: one thread block if room
            std::vector<DevOp> in, thr;
            for (auto &d : all) {
                if (in_tile_diag(d) && !(tm(d) & F.rmask)) thr.push_back(d);
                else in.push_back(d);
            }
            int thr_off = -1;
            if (!thr.empty()) {
                thr_off = take_block(1);
                if (thr_off < 0) {
                    in = all;
                    thr.clear();
                }
            }
            const int N = (int)in.size();
            std::vector<uint32_t> m(N);
            std::vector<char> dg(N), ry(N), done(N, 0);
            for (int i = 0; i < N; ++i) {
                m[i] = tm(in[i]);
                dg[i] = diag_kind(in[i].kind);
                ry[i] = in[i].kind == SV_RY && in[i].t[0] < kOutTarget && (F.rmask >> in[i].t[0] & 1u);
            }
            std::vector<int> npred(N, 0);
            std::vector<std::vector<int>> succ(N);
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < j; ++i)
                    if ((m[i] & m[j]) && !(dg[i] && dg[j])) {
                        ++npred[j];
                        succ[i].push_back(j);
                    }
            std::vector<DevOp> out;
            auto regidx = [&](int t) { return __builtin_popcount(F.rmask & ((1u << t) - 1u)); };
            auto emit_op = [&](const DevOp &d) { out.push_back(d); };
            auto emit = [&](int i) {
                done[i] = 1;
                for (int j : succ[i]) --npred[j];
                emit_op(in[i]);
            };
            auto push_op = [&](int i) {
                RegStep st;
                st.type = SV_STEP_OP;
                st.op_begin = F.op_begin + (int32_t)out.size();
                st.op_end = st.op_begin + 1;
                st.a = st.op_begin;
                emit(i);
                P.steps.push_back(st);
            };
            auto member = [&](const DevOp &d, int pos) {
                DiagMember dm;
                dm.op = F.op_begin + pos;
                dm.a = dm.b = 0;
                if (d.kind == SV_RZ) {
                    const int t = d.t[0];
                    if (F.rmask >> t & 1u) { dm.type = SV_DM_REG_RZ; dm.a = regidx(t); }
                    else { dm.type = SV_DM_THR_RZ; dm.a = t; }
                } else {
                    const int t0 = d.t[0], t1 = d.t[1];
                    const bool r0 = F.rmask >> t0 & 1u, r1 = F.rmask >> t1 & 1u;
                    if (r0 && r1) { dm.type = SV_DM_REG_CZ; dm.a = regidx(t0); dm.b = regidx(t1); }
                    else if (!r0 && !r1) { dm.type = SV_DM_THR_CZ; dm.a = t0; dm.b = t1; }
                    else { dm.type = SV_DM_MIX_CZ; dm.a = regidx(r0 ? t0 : t1); dm.b = r0 ? t1 : t0; }
                }
                return dm;
            };
            // emits a block of the given ops (positions follow in `out`)
            auto push_block = [&](int kind, int off, const std::vector<DevOp> &ops, const std::vector<int> &idx) {
                const int bi = (int)P.dblocks.size();
                DiagBlock B;
                B.op_begin = F.op_begin + (int32_t)out.size();
                B.m_begin = (int32_t)P.dmembers.size();
                B.rmask = F.rmask;
                B.kind = kind;
                B.smem = off;
                B.lanes = F.lanes;
                for (size_t u = 0; u < ops.size(); ++u) {
                    P.dmembers.push_back(member(ops[u], (int)out.size()));
                    if (idx.empty()) emit_op(ops[u]);
                    else emit(idx[u]);
                    out.back().mat = -2 - bi;
                }
                B.op_end = F.op_begin + (int32_t)out.size();
                B.m_end = (int32_t)P.dmembers.size();
                P.dblocks.push_back(B);
                RegStep st;
                st.type = SV_STEP_DIAG;
                st.a = bi;
                st.op_begin = B.op_begin;
                st.op_end = B.op_end;
                P.steps.push_back(st);
            };
            int left = N;
            while (left > 0) {
                std::vector<int> rys, others, diags;
                for (int i = 0; i < N; ++i) {
                    if (done[i] || npred[i]) continue;
                    if (ry[i]) rys.push_back(i);
                    else if (dg[i]) diags.push_back(i);
                    else others.push_back(i);
                }
                if (!rys.empty()) {
                    std::sort(rys.begin(), rys.end(), [&](int a, int b) { return in[a].t[0] < in[b].t[0]; });
                    RegStep st;
                    st.type = SV_STEP_ROT;
                    st.op_begin = F.op_begin + (int32_t)out.size();
                    st.a = 0;
                    for (int i : rys) {
                        st.a |= 1 << regidx(in[i].t[0]);
                        emit(i);
                    }
                    st.op_end = F.op_begin + (int32_t)out.size();
                    P.steps.push_back(st);
                    left -= (int)rys.size();
                    continue;
                }
                if (!others.empty()) {
                    for (int i : others) push_op(i);
                    left -= (int)others.size();
                    continue;
                }
                // diagonal operations only: blockable ones as one run, the rest one by one
                std::vector<int> run;
                for (int i : diags) {
                    const DevOp &d = in[i];
                    // a thread-only member cannot go into a register block
                    if (in_tile_diag(d) && (tm(d) & F.rmask)) run.push_back(i);
                    else push_op(i);
                }
                left -= (int)diags.size();
                if (run.empty()) continue;
                std::vector<DevOp> rops;
                for (int i : run) rops.push_back(in[i]);
                const int off = diag_run_pays(rops) ? take_block(0) : -1;
                if (off < 0) {
                    for (int i : run) push_op(i);
                    continue;
                }
                push_block(0, off, rops, run);
            }
            if (!thr.empty()) push_block(1, thr_off, thr, {});
            std::copy(out.begin(), out.end(), P.ops.begin() + F.op_begin);
            F.st_end = (int32_t)P.steps.size();
        }
        gp.db_end = (int32_t)P.dblocks.size();
        gp.st_begin = P.phases[gp.ph_begin].st_begin;
        gp.st_end = P.phases[gp.ph_end - 1].st_end;
        gp.area = area;
        gp.mem_begin = gp.db_end > gp.db_begin ? P.dblocks[gp.db_begin].m_begin : 0;
        gp.mem_end = gp.db_end > gp.db_begin ? P.dblocks[gp.db_end - 1].m_end : 0;
    }
}

// ---------------------------------------------------------- coset passes --
// Strings sharing a physical X/Y mask x form a group: one read of psi serves
// all of them.  A pass stages 2^(kl+m) amplitudes: the 2^m runs of 2^kl
// contiguous amplitudes at rep ^ span(a), a in [0, 2^m), for one coset
// representative rep of an m-dimensional span V over bits >= kl.  Every group
// whose high part x >> kl lies in V pairs amplitudes inside the staged set, so
// all such groups share the pass.  Per pass: the span is chosen at the
// shortest run (largest span) by two greedy rules -- V spanned by single bits
// (Alg. 3-like, lightest masks first) or by the most frequent masks -- and the
// one covering more strings is kept; then the run is lengthened as far as the
// staged size allows (projecting the span onto the bits above the run keeps
// every selected group covered) and the span is padded with the lowest free
// bits so that every pass stages the same amount.
struct GroupIn {
    uint64_t x;
    std::vector<std::pair<uint64_t, double>> zs;   // unique z with summed coefficient
    std::vector<std::vector<int32_t>> terms;       // input terms per z
};

struct Span {
    std::vector<uint64_t> basis;
    std::vector<int32_t> pivot;
    uint64_t reduce(uint64_t r) const {
        for (size_t j = 0; j < basis.size(); ++j)
            if (r >> pivot[j] & 1) r ^= basis[j];
        return r;
    }
    void insert(uint64_t v) {
        v = reduce(v);
        if (!v) return;
        const int p = hibit(v);
        for (auto &b : basis)
            if (b >> p & 1) b ^= v;
        basis.push_back(v);
        pivot.push_back(p);
    }
};

void plan_cosets(EvcPlan &P, std::vector<GroupIn> &groups, int klmin, int mmax, int klmax, uint64_t allowed) {
    // runs stay inside the contiguous low allowed bits (local bits for EVC)
    int lowallowed = 0;
    while (lowallowed < 64 && (allowed >> lowallowed & 1)) ++lowallowed;
    const int stage = std::min(klmin, lowallowed) + mmax;
    klmin = std::min(klmin, lowallowed);
    klmax = std::min(klmax, lowallowed);
    const uint64_t lowmin = bit(klmin) - 1;
    std::vector<int32_t> remaining(groups.size());
    std::iota(remaining.begin(), remaining.end(), 0);
    while (!remaining.empty()) {
        auto run = [&](bool bits_mode, Span &sp, std::vector<int32_t> &sel) {
            sp = Span();
            sel.clear();
            if (bits_mode) {
                std::vector<int32_t> byw(remaining);
                std::stable_sort(byw.begin(), byw.end(), [&](int32_t a, int32_t b) {
                    return popc(groups[a].x & ~lowmin) < popc(groups[b].x & ~lowmin);
                });
                uint64_t B = 0;
                for (int32_t gi : byw) {
                    const uint64_t h = groups[gi].x & ~lowmin & allowed;
                    if (popc(B | h) <= mmax) B |= h;
                    if (popc(B) == mmax) break;
                }
                for (uint64_t v = B; v; v &= v - 1) sp.insert(bit(lobit(v)));
            } else {
                while ((int)sp.basis.size() < mmax) {
                    std::unordered_map<uint64_t, int64_t> freq;
                    uint64_t best = 0;
                    int64_t bestc = 0;
                    for (int32_t gi : remaining) {
                        const uint64_t r = sp.reduce(groups[gi].x & ~lowmin);
                        if (!r) continue;
                        const int64_t c = (freq[r] += (int64_t)groups[gi].zs.size());
                        if (c > bestc) { bestc = c; best = r; }
                    }
                    if (!best) break;
                    sp.insert(best);
                }
            }
            int64_t strings = 0;
            for (int32_t gi : remaining) {
                if (sp.reduce(groups[gi].x & ~lowmin)) continue;
                const int64_t c = (int64_t)groups[gi].zs.size();
                if (strings + c > kMaxPassStrings && !sel.empty()) continue;
                sel.push_back(gi);
                strings += c;
            }
            return strings;
        };
        Span sA, sB;
        std::vector<int32_t> selA, selB;
        const int64_t cA = run(true, sA, selA);
        const int64_t cB = run(false, sB, selB);
        const bool useA = cA >= cB;
        const Span &chosen = useA ? sA : sB;
        const std::vector<int32_t> &sel = useA ? selA : selB;
        // lengthen the run as far as the staged size allows
        const int kl = std::max(klmin, std::min(klmax, stage - (int)chosen.basis.size()));
        const uint64_t lowmask = bit(kl) - 1;
        Span sp;
        for (uint64_t v : chosen.basis) sp.insert(v & ~lowmask);
        uint64_t pivmask = 0;
        for (int32_t pv : sp.pivot) pivmask |= bit(pv);
        for (int b = kl; b < 64 && (int)sp.basis.size() < stage - kl; ++b) {
            if (!(allowed >> b & 1) || (pivmask >> b & 1)) continue;
            for (auto &v : sp.basis)
                if (v >> b & 1) v ^= bit(b);
            sp.basis.push_back(bit(b));
            sp.pivot.push_back(b);
            pivmask |= bit(b);
        }
        CosetPass cp;
        cp.kl = kl;
        cp.m = (int32_t)sp.basis.size();
        for (int j = 0; j < cp.m; ++j) { cp.basis[j] = sp.basis[j]; cp.pivot[j] = sp.pivot[j]; }
        cp.g_begin = (int32_t)P.groups.size();
        cp.s_begin = (int32_t)P.strings.size();
        std::vector<char> in(groups.size(), 0);
        for (int32_t gi : sel) {
            in[gi] = 1;
            GroupIn &G = groups[gi];
            EvcGroup eg;
            eg.x = G.x;
            uint32_t c = 0;
            const uint64_t h = G.x & ~lowmask;
            for (int j = 0; j < cp.m; ++j)
                if (h >> sp.pivot[j] & 1) c |= 1u << j;
            eg.X = (c << kl) | (uint32_t)(G.x & lowmask);
            eg.s_begin = (int32_t)P.strings.size();
            for (size_t s = 0; s < G.zs.size(); ++s) {
                EvcString es;
                es.z = G.zs[s].first;
                es.nY = popc(G.x & G.zs[s].first) & 3;
                es.coef = G.zs[s].second;
                es.bz = 0;
                for (int j = 0; j < cp.m; ++j)
                    if (popc(sp.basis[j] & es.z) & 1) es.bz |= 1u << j;
                for (int32_t t : G.terms[s]) P.term_slot[t] = (int32_t)P.strings.size();
                P.strings.push_back(es);
            }
            eg.s_end = (int32_t)P.strings.size();
            P.groups.push_back(eg);
        }
        cp.g_end = (int32_t)P.groups.size();
        cp.s_end = (int32_t)P.strings.size();
        P.passes.push_back(cp);
        std::vector<int32_t> next;
        for (int32_t gi : remaining)
            if (!in[gi]) next.push_back(gi);
        remaining.swap(next);
    }
}

void group_terms(const std::vector<int32_t> &terms, const sv_pauli *p, const double *coeffs,
                 const std::vector<int32_t> &l2p, std::vector<GroupIn> &groups) {
    std::unordered_map<uint64_t, int32_t> gidx;
    for (int32_t t : terms) {
        uint64_t x = to_physical(p[t].x, l2p), z = to_physical(p[t].z, l2p);
        // a group holds at most kMaxGroupStrings distinct z; a full group for
        // this x is closed and a new one (same x) opened
        auto it = gidx.find(x);
        int32_t gi;
        if (it == gidx.end()) {
            gi = (int32_t)groups.size();
            gidx[x] = gi;
            groups.push_back(GroupIn{x, {}, {}});
        } else {
            gi = it->second;
        }
        size_t s = 0;
        while (s < groups[gi].zs.size() && groups[gi].zs[s].first != z) ++s;
        if (s == groups[gi].zs.size() && s >= (size_t)kMaxGroupStrings) {
            gi = (int32_t)groups.size();
            gidx[x] = gi;
            groups.push_back(GroupIn{x, {}, {}});
            s = 0;
        }
        GroupIn &G = groups[gi];
        if (s == G.zs.size()) {
            G.zs.push_back({z, 0.0});
            G.terms.push_back({});
        }
        G.zs[s].second += coeffs ? coeffs[t] : 0.0;
        G.terms[s].push_back(t);
    }
}

// Lexicographic rank of k-combinations of {0..n-1} via binomial sums.
struct Binom {
    std::vector<std::vector<int64_t>> C;
    explicit Binom(int n) : C(n + 2, std::vector<int64_t>(n + 2, 0)) {
        for (int a = 0; a <= n + 1; ++a) {
            C[a][0] = 1;
            for (int b = 1; b <= a; ++b) C[a][b] = C[a - 1][b - 1] + (b <= a - 1 ? C[a - 1][b] : 0);
        }
    }
    int64_t operator()(int a, int b) const {
        if (a < 0 || b < 0 || b > a) return 0;
        return C[a][b];
    }
};

// Visit every k-subset of `free` (ascending) with its lexicographic rank
// among the k-subsets of {0..n-1}.
template <class F>
void for_each_subset_rank(const std::vector<int> &fr, int k, int n, const Binom &B, F &&f) {
    if (k == 0) { f(0); return; }
    std::vector<int> idx(k);
    std::vector<int64_t> acc(k + 1, 0);
    // term for position i with value c given previous value pc:
    //   C(n - pc - 1, k - i) - C(n - c, k - i)
    int m = (int)fr.size();
    if (m < k) return;
    int i = 0;
    idx[0] = 0;
    while (true) {
        if (idx[i] <= m - (k - i)) {
            int pc = (i == 0) ? -1 : fr[idx[i - 1]];
            int c = fr[idx[i]];
            acc[i + 1] = acc[i] + B(n - pc - 1, k - i) - B(n - c, k - i);
            if (i == k - 1) {
                f(acc[k]);
                ++idx[i];
            } else {
                idx[i + 1] = idx[i] + 1;
                ++i;
            }
        } else {
            if (i == 0) break;
            --i;
            ++idx[i];
        }
    }
}

// Alg. 6 with diagonalization: targets are X/Y supports; identical supports
// merged with multiplicity; each step takes the first global set (in
// lexicographic order) whose complement holds the most remaining strings.
// Counts are maintained incrementally: a support x adds its multiplicity to
// every global set disjoint from it.
std::string tiling_pauli_strings(int n, int nG, const sv_pauli *p, const std::vector<int32_t> &terms,
                                 const PlanOptions &o, std::vector<std::vector<int32_t>> &tiles_terms,
                                 std::vector<uint64_t> &tiles_local) {
    const uint64_t Q = bit(n) - 1;
    std::unordered_map<uint64_t, int32_t> xi;
    std::vector<uint64_t> xs;
    std::vector<std::vector<int32_t>> members;
    for (int32_t t : terms) {
        uint64_t x = p[t].x;
        if (popc(x) > n - nG) return "a Pauli string has more X/Y positions than local qubits";
        auto it = xi.find(x);
        if (it == xi.end()) {
            xi[x] = (int32_t)xs.size();
            xs.push_back(x);
            members.push_back({t});
        } else {
            members[it->second].push_back(t);
        }
    }
    Binom B(n);
    int64_t ncand = B(n, nG);
    auto unrank = [&](int64_t r) {
        uint64_t G = 0;
        int c = 0;
        for (int i = 0; i < nG; ++i) {
            while (true) {
                int64_t cnt = B(n - c - 1, nG - i - 1);
                if (r < cnt) break;
                r -= cnt;
                ++c;
            }
            G |= bit(c);
            ++c;
        }
        return G;
    };
    if (o.alg6_step) {
        // greedy steps on the device: counts recomputed per step, no table
        std::vector<int32_t> w(xs.size());
        for (size_t gi = 0; gi < xs.size(); ++gi) w[gi] = (int32_t)members[gi].size();
        size_t left = xs.size();
        while (left) {
            int64_t bestr = -1, best = 0;
            std::string e = o.alg6_step(xs, w, n, nG, bestr, best);
            if (!e.empty()) return e;
            if (best <= 0 || bestr < 0 || bestr >= ncand) return "no mapping holds a remaining Pauli string";
            const uint64_t G = unrank(bestr);
            std::vector<int32_t> tile;
            for (size_t gi = 0; gi < xs.size(); ++gi) {
                if (!w[gi] || (xs[gi] & G)) continue;
                w[gi] = 0;
                --left;
                tile.insert(tile.end(), members[gi].begin(), members[gi].end());
            }
            std::sort(tile.begin(), tile.end());
            tiles_terms.push_back(tile);
            tiles_local.push_back(Q & ~G);
        }
        return "";
    }
    if (ncand > 60000000) return "Alg. 6 search space C(n, n_G) too large for the host search";
    std::vector<int64_t> count((size_t)ncand, 0);
    auto add = [&](size_t gi, int64_t w) {
        std::vector<int> fr;
        for (uint64_t v = Q & ~xs[gi]; v; v &= v - 1) fr.push_back(lobit(v));
        for_each_subset_rank(fr, nG, n, B, [&](int64_t r) { count[(size_t)r] += w; });
    };
    for (size_t gi = 0; gi < xs.size(); ++gi) add(gi, (int64_t)members[gi].size());
    std::vector<char> alive(xs.size(), 1);
    size_t left = xs.size();
    while (left) {
        int64_t best = 0, bestr = -1;
        for (int64_t r = 0; r < ncand; ++r)
            if (best < count[(size_t)r]) { best = count[(size_t)r]; bestr = r; }
        if (bestr < 0) return "no mapping holds a remaining Pauli string";
        const uint64_t G = unrank(bestr);
        std::vector<int32_t> tile;
        for (size_t gi = 0; gi < xs.size(); ++gi) {
            if (!alive[gi] || (xs[gi] & G)) continue;
            alive[gi] = 0;
            --left;
            tile.insert(tile.end(), members[gi].begin(), members[gi].end());
            add(gi, -(int64_t)members[gi].size());
        }
        std::sort(tile.begin(), tile.end());
        tiles_terms.push_back(tile);
        tiles_local.push_back(Q & ~G);
    }
    return "";
}

}  // namespace

uint64_t hash_bytes(const void *p, size_t n, uint64_t h) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string validate_gates(int n, const sv_gate *gates, size_t m, size_t np, size_t nmats) {
    for (size_t i = 0; i < m; ++i) {
        const sv_gate &g = gates[i];
        int nq = gate_nq(g.kind);
        if (nq < 0) return "gate " + std::to_string(i) + ": unknown kind";
        uint64_t seen = 0;
        for (int t = 0; t < 4; ++t) {
            if (t < nq) {
                if (g.q[t] < 0 || g.q[t] >= n) return "gate " + std::to_string(i) + ": qubit out of range";
                if (seen & bit(g.q[t])) return "gate " + std::to_string(i) + ": duplicate target";
                seen |= bit(g.q[t]);
            }
        }
        bool parametric = g.kind == SV_RY || g.kind == SV_RZ || g.kind == SV_GIVENS || g.kind == SV_DEXC;
        if (parametric && (g.param < 0 || (size_t)g.param >= np))
            return "gate " + std::to_string(i) + ": parameter index out of range";
        if (g.kind >= SV_MAT1 && nmats != (size_t)-1) {   // (size_t)-1: planning only, no matrices
            size_t dim = (size_t)1 << nq;
            if (g.mat < 0 || (size_t)g.mat + dim * dim > nmats)
                return "gate " + std::to_string(i) + ": matrix out of range";
        }
    }
    return "";
}

std::string plan_qsu(int n, int g, const sv_gate *gates, size_t m, bool lazy, const PlanOptions &o,
                     const std::vector<int32_t> &l2p_init, QsuPlan &P) {
    P = QsuPlan();
    P.n = n; P.g = g; P.nL = n - g;
    std::vector<Op> ops(m);
    for (size_t i = 0; i < m; ++i) {
        Op &op = ops[i];
        op.kind = gates[i].kind;
        op.nq = gate_nq(op.kind);
        for (int t = 0; t < op.nq; ++t) {
            op.q[t] = gates[i].q[t];
            op.tmask |= bit(op.q[t]);
        }
        op.param = gates[i].param;
        op.mat = gates[i].mat;
        if (op.nq > P.nL) return "an operator is wider than the local qubits";
    }
    P.init_l2p = l2p_init;
    std::string err;
    if (lazy && o.hier_intra >= 0) {
        if (o.hier_intra > g) return "more intra qubits than global qubits";
        err = hierarchical_tiling(n, P.nL, o.hier_intra, ops, o.pad_highest, l2p_init, P.order, P.tiles,
                                  P.final_l2p);
    } else if (lazy) {
        err = flat_tiling(n, P.nL, ops, o.pad_highest, l2p_init, P.order, P.tiles, P.final_l2p, o.diag_exempt);
    } else {
        err = adhoc_schedule(n, P.nL, ops, depth_sort(ops), l2p_init, P.order, P.tiles, P.final_l2p);
    }
    if (!err.empty()) return err;
    if (P.tiles.empty()) P.final_l2p = l2p_init;
    int k = std::max(o.tile_bits, std::min(o.low_bits, P.nL) + 4);
    plan_gate_passes(P, ops, k, o.low_bits, o.fuse_max, o.diag_exempt);
    plan_phases(P, o.reg_pairs);
    plan_steps(P, std::min(o.max_diag, kMaxPassDiag), o.amp_bytes);
    return "";
}

std::string plan_evc(int n, int g, const sv_pauli *p, const double *coeffs, size_t nterms, bool lazy,
                     const PlanOptions &o, const std::vector<int32_t> &l2p_init, EvcPlan &P) {
    P = EvcPlan();
    P.n = n; P.g = g; P.nL = n - g;
    P.init_l2p = l2p_init;
    P.term_slot.assign(nterms, -1);
    std::vector<int32_t> l2p = l2p_init;
    uint64_t cur = local_set(l2p, P.nL);
    // strings whose X/Y support exceeds n_L fit no mapping: they are kept for
    // one last tile without a QR whose amplitude pairs cross chunks
    std::vector<int32_t> narrow, wide;
    for (size_t t = 0; t < nterms; ++t) (popc(p[t].x) > P.nL ? wide : narrow).push_back((int32_t)t);
    std::vector<std::vector<int32_t>> tt;
    std::vector<uint64_t> tl;
    if (lazy) {
        std::string err = tiling_pauli_strings(n, g, p, narrow, o, tt, tl);
        if (!err.empty()) return err;
        for (size_t i = 0; i < tt.size(); ++i) {
            Tile t;
            t.begin = (int32_t)P.order.size();
            P.order.insert(P.order.end(), tt[i].begin(), tt[i].end());
            t.end = (int32_t)P.order.size();
            t.local_mask = tl[i];
            if (tl[i] != cur) qr_pairs(l2p, cur, tl[i], t.pairs);
            cur = tl[i];
            t.l2p = l2p;
            P.tiles.push_back(std::move(t));
        }
    } else {
        // targets: full support when it fits n_L qubits, else the X/Y support
        std::vector<uint64_t> tms(nterms);
        for (size_t t = 0; t < nterms; ++t) {
            uint64_t full = p[t].x | p[t].z;
            tms[t] = popc(full) <= P.nL ? full : p[t].x;
        }
        // the ad hoc rule on masks (a string may have more than 4 targets)
        uint64_t QL = cur;
        std::vector<int64_t> last(n, -1);
        Tile ct;
        ct.begin = 0;
        ct.local_mask = QL;
        ct.l2p = l2p;
        for (size_t xi = 0; xi < narrow.size(); ++xi) {
            const int32_t term = narrow[xi];
            uint64_t t = tms[term];
            if (t & ~QL) {
                uint64_t inn = t & ~QL;
                int k = popc(inn);
                std::vector<int32_t> cand;
                for (uint64_t v = QL & ~t; v; v &= v - 1) cand.push_back(lobit(v));
                std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
                    if (last[a] != last[b]) return last[a] < last[b];
                    return a > b;
                });
                uint64_t ev = 0;
                for (int i = 0; i < k; ++i) ev |= bit(cand[i]);
                uint64_t nQL = (QL & ~ev) | inn;
                if ((int32_t)P.order.size() > ct.begin) {
                    ct.end = (int32_t)P.order.size();
                    P.tiles.push_back(ct);
                }
                ct = Tile();
                ct.begin = (int32_t)P.order.size();
                qr_pairs(l2p, QL, nQL, ct.pairs);
                QL = nQL;
                ct.local_mask = QL;
                ct.l2p = l2p;
            }
            P.order.push_back(term);
            for (uint64_t v = t; v; v &= v - 1) last[lobit(v)] = (int64_t)xi;
        }
        if ((int32_t)P.order.size() > ct.begin) {
            ct.end = (int32_t)P.order.size();
            P.tiles.push_back(ct);
        }
        cur = QL;
    }
    P.tile_wide.assign(P.tiles.size(), 0);
    if (!wide.empty()) {
        Tile t;
        t.begin = (int32_t)P.order.size();
        P.order.insert(P.order.end(), wide.begin(), wide.end());
        t.end = (int32_t)P.order.size();
        t.local_mask = local_set(l2p, P.nL);
        t.l2p = l2p;
        P.tiles.push_back(std::move(t));
        P.tile_wide.push_back(1);
    }
    P.final_l2p = l2p;
    if (P.tiles.empty()) P.final_l2p = l2p_init;
    const int klmin = std::min(o.evc_low_bits, P.nL);
    const int mmax = std::min(o.evc_span, kMaxSpan);
    const int klmax = std::max(klmin, kMaxRunBits);
    const uint64_t localbits = bit(P.nL) - 1;
    const uint64_t allbits = bit(n) - 1;
    for (size_t ti = 0; ti < P.tiles.size(); ++ti) {
        const Tile &T = P.tiles[ti];
        std::vector<int32_t> terms(P.order.begin() + T.begin, P.order.begin() + T.end);
        std::vector<GroupIn> groups;
        group_terms(terms, p, coeffs, T.l2p, groups);
        P.tile_pass_begin.push_back((int32_t)P.passes.size());
        plan_cosets(P, groups, klmin, mmax, klmax, P.tile_wide[ti] ? allbits : localbits);
        P.tile_pass_end.push_back((int32_t)P.passes.size());
    }
    return "";
}

std::string plan_hpsi(int n, const sv_pauli *p, const double *coeffs, size_t nterms, const PlanOptions &o,
                      const std::vector<int32_t> &l2p, EvcPlan &P) {
    P = EvcPlan();
    P.n = n; P.g = 0; P.nL = n;
    P.init_l2p = l2p;
    P.final_l2p = l2p;
    P.term_slot.assign(nterms, -1);
    Tile t;
    t.begin = 0;
    for (size_t i = 0; i < nterms; ++i) P.order.push_back((int32_t)i);
    t.end = (int32_t)nterms;
    t.local_mask = bit(n) - 1;
    t.l2p = l2p;
    P.tiles.push_back(t);
    std::vector<GroupIn> groups;
    group_terms(P.order, p, coeffs, l2p, groups);
    P.tile_pass_begin.push_back(0);
    plan_cosets(P, groups, std::min(o.evc_low_bits, n), std::min(o.evc_span, kMaxSpan),
                std::max(std::min(o.evc_low_bits, n), kMaxRunBits), bit(n) - 1);
    P.tile_pass_end.push_back((int32_t)P.passes.size());
    return "";
}

void permutation_swaps(const std::vector<int32_t> &from, const std::vector<int32_t> &to,
                       std::vector<std::vector<int32_t>> &sets) {
    int n = (int)from.size();
    std::vector<int32_t> pi(n, -1);            // physical bit p (layout from) -> physical bit in `to`
    for (int q = 0; q < n; ++q) pi[from[q]] = to[q];
    std::vector<int32_t> A, Bs;
    std::vector<char> seen(n, 0);
    for (int s = 0; s < n; ++s) {
        if (seen[s] || pi[s] == s) { seen[s] = 1; continue; }
        std::vector<int32_t> cyc;
        for (int c = s; !seen[c]; c = pi[c]) { seen[c] = 1; cyc.push_back(c); }
        int k = (int)cyc.size();
        // A: c_i <-> c_{-i};  B: c_i <-> c_{1-i}; B o A maps c_i -> c_{i+1}
        for (int i = 1; i < k; ++i) {
            int j = (k - i) % k;
            if (i < j) { A.push_back(cyc[i]); A.push_back(cyc[j]); }
        }
        for (int i = 0; i < k; ++i) {
            int j = ((1 - i) % k + k) % k;
            if (i < j) { Bs.push_back(cyc[i]); Bs.push_back(cyc[j]); }
        }
    }
    sets.clear();
    if (!A.empty()) sets.push_back(A);
    if (!Bs.empty()) sets.push_back(Bs);
}

}  // namespace sv
