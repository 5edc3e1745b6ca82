// Device kernels of the hot path (sm_103a).
//
//   k_gate_pass   K-GATE: stage 2^k amplitudes of a tile in shared memory,
//                 apply a whole pass of narrow gates (Eq. apply_parallel:
//                 every virtual chunk applies the same local operator), store.
//   k_adj_pass    K-ADJ: the same tiles of psi and lambda; per gate, in reverse,
//                 the partial of Im<lambda|G|psi> and then U^dagger on both.
//   k_bitswap     K-QR: in-place exchange of physical index bit pairs (the
//                 qubit reordering of Sec. III-B-4: two elements whose indices
//                 differ only at the paired bits are swapped).
//   k_evc_pass    K-EVC: <psi|P|psi> for all strings whose X/Y mask pairs
//                 amplitudes inside one staged coset (Eqs. evc, parallel_evc,
//                 par_exp).
//   k_hpsi_pass   K-HPSI: lambda += sum_t a_t P_t psi over the same cosets.
//   k_reduce_rows K-RED: fixed-order FP64 reduction of per-CTA partials.
//
// All kernels are persistent grid-stride loops over independent work units
// (tiles or cosets); a CTA never waits on another CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "kernels.h"

namespace sv {
namespace {

template <typename R> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };
template <typename R> using Cx = typename CxT<R>::T;

template <typename R>
__device__ __forceinline__ Cx<R> mk(R a, R b) {
    Cx<R> c;
    c.x = a;
    c.y = b;
    return c;
}

__device__ __forceinline__ uint32_t ins0(uint32_t p, int b) {
    return ((p >> b) << (b + 1)) | (p & ((1u << b) - 1u));
}

__device__ __forceinline__ uint64_t deposit(uint64_t v, const int8_t *bits, int nb) {
    uint64_t o = 0;
    for (int i = 0; i < nb; ++i) o |= ((v >> i) & 1ull) << bits[i];
    return o;
}

// Stepping deposit(v) to deposit(v + stride) without re-depositing: with the
// bit list ascending, deposit is an order-preserving embedding, so the sum is
// the masked addition ((x | ~mask) + deposit(stride)) & mask (carries ripple
// through the bits outside the mask).
struct BitWalk {
    uint64_t nmask, d;
};
__device__ __forceinline__ BitWalk bit_walk(const int8_t *bits, int nb, uint64_t stride) {
    uint64_t m = 0;
    for (int i = 0; i < nb; ++i) m |= 1ull << bits[i];
    return {~m, deposit(stride, bits, nb)};
}
__device__ __forceinline__ uint64_t walk_next(uint64_t x, const BitWalk &w) {
    return ((x | w.nmask) + w.d) & ~w.nmask;
}

template <typename R>
__device__ __forceinline__ void rot(Cx<R> &u, Cx<R> &v, R c, R s) {
    const Cx<R> a = u, b = v;
    u = mk<R>(c * a.x - s * b.x, c * a.y - s * b.y);
    v = mk<R>(s * a.x + c * b.x, s * a.y + c * b.y);
}

// complex64: the same rotation on packed pairs (one f32x2 instruction per
// real and imaginary part together; same rounding: one rounded product, then
// a fused multiply-add)
__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
// the rotation with the coefficient pairs (c, c), (s, s), (-s, -s) already packed
struct RotPairs {
    unsigned long long C, S, NS;
};
__device__ __forceinline__ RotPairs rot_pairs(float c, float s) {
    return {f2_pack(c, c), f2_pack(s, s), f2_pack(-s, -s)};
}
__device__ __forceinline__ void rot_packed(float2 &u, float2 &v, const RotPairs &k) {
    const unsigned long long U = f2_pack(u.x, u.y), V = f2_pack(v.x, v.y);
    unsigned long long t, uu, vv;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(V), "l"(k.NS));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(uu) : "l"(U), "l"(k.C), "l"(t));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(V), "l"(k.C));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(vv) : "l"(U), "l"(k.S), "l"(t));
    u = f2_unpack(uu);
    v = f2_unpack(vv);
}
template <>
__device__ __forceinline__ void rot<float>(float2 &u, float2 &v, float c, float s) {
    rot_packed(u, v, rot_pairs(c, s));
}

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Matrix element (row i, column j) of a dim x dim complex matrix, or of its
// conjugate transpose.
template <typename R>
__device__ __forceinline__ Cx<R> mel(const Cx<R> *M, int dim, int i, int j, bool adj) {
    if (!adj) return M[i * dim + j];
    Cx<R> v = M[j * dim + i];
    return mk<R>(v.x, -v.y);
}

template <typename R, int NQ>
__device__ __forceinline__ void dense_group(Cx<R> *t, const uint32_t *idx, const Cx<R> *M, bool adj) {
    constexpr int D = 1 << NQ;
    Cx<R> in[D];
#pragma unroll
    for (int j = 0; j < D; ++j) in[j] = t[idx[j]];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        R re = 0, im = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            Cx<R> m = mel<R>(M, D, i, j, adj);
            re += m.x * in[j].x - m.y * in[j].y;
            im += m.x * in[j].y + m.y * in[j].x;
        }
        t[idx[i]] = mk<R>(re, im);
    }
}

// Sort up to 4 small ints ascending (insertion sort).
__device__ __forceinline__ void sort4(int *s, int n) {
    for (int i = 1; i < n; ++i) {
        int v = s[i], j = i - 1;
        while (j >= 0 && s[j] > v) { s[j + 1] = s[j]; --j; }
        s[j + 1] = v;
    }
}

// Caller matrices (MAT1/2/4), kept out of line so that their 16-element
// register arrays do not inflate the register allocation of the gate loops.
template <typename R>
__device__ __noinline__ void apply_dense_op(Cx<R> *t, int k, const DevOp op, const Cx<R> *mats, bool adj) {
    const uint32_t T = 1u << k;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    switch (op.kind) {
    case SV_MAT1: {
        const Cx<R> *M = mats + op.mat;
        const int b = op.t[0];
        for (uint32_t p = tid; p < T / 2; p += nt) {
            uint32_t idx[2];
            idx[0] = ins0(p, b);
            idx[1] = idx[0] | (1u << b);
            dense_group<R, 1>(t, idx, M, adj);
        }
        break;
    }
    case SV_MAT2: {
        const Cx<R> *M = mats + op.mat;
        const int lo = min((int)op.t[0], (int)op.t[1]), hi = max((int)op.t[0], (int)op.t[1]);
        for (uint32_t p = tid; p < T / 4; p += nt) {
            const uint32_t base = ins0(ins0(p, lo), hi);
            uint32_t idx[4];
            for (int j = 0; j < 4; ++j)
                idx[j] = base | ((j & 1) ? (1u << op.t[0]) : 0u) | ((j & 2) ? (1u << op.t[1]) : 0u);
            dense_group<R, 2>(t, idx, M, adj);
        }
        break;
    }
    case SV_MAT4: {
        const Cx<R> *M = mats + op.mat;
        int srt[4] = {op.t[0], op.t[1], op.t[2], op.t[3]};
        sort4(srt, 4);
        for (uint32_t p = tid; p < T / 16; p += nt) {
            uint32_t base = p;
            for (int i = 0; i < 4; ++i) base = ins0(base, srt[i]);
            uint32_t idx[16];
            for (int j = 0; j < 16; ++j) {
                uint32_t o = base;
                for (int q = 0; q < 4; ++q)
                    if (j >> q & 1) o |= 1u << op.t[q];
                idx[j] = o;
            }
            dense_group<R, 4>(t, idx, M, adj);
        }
        break;
    }
    default:
        break;
    }
}

// Apply one narrow gate to a staged tile of 2^k amplitudes (tile-local bit
// positions in op.t).  U = exp(-i theta G/2); adj applies U^dagger.
// Each thread owns whole index groups, so the caller syncs between gates.
// Diagonal gates on qubits outside the staged tile (diagonal exemption)
// become, for one tile, one of these operations: a phase on the whole tile
// (RZ; t[0] = the qubit's bit in this tile), Z on an in-tile bit t[0] (CZ
// whose outside qubit is 1 here), -1 on the whole tile (CZ of two outside
// qubits that are both 1), or nothing.
enum { SV_OP_PHASE = 100, SV_OP_ZSIGN = 101, SV_OP_NEG = 102, SV_OP_NOP = 103 };

__device__ __forceinline__ DevOp resolve_out(DevOp op, uint64_t gbase) {
    if (op.kind == SV_RZ && op.t[0] >= kOutTarget) {
        op.t[0] = (int8_t)((gbase >> (op.t[0] - kOutTarget)) & 1ull);
        op.kind = SV_OP_PHASE;
    } else if (op.kind == SV_CZ && (op.t[0] >= kOutTarget || op.t[1] >= kOutTarget)) {
        const bool o0 = op.t[0] >= kOutTarget, o1 = op.t[1] >= kOutTarget;
        const int b0 = o0 ? (int)((gbase >> (op.t[0] - kOutTarget)) & 1ull) : 0;
        const int b1 = o1 ? (int)((gbase >> (op.t[1] - kOutTarget)) & 1ull) : 0;
        if (o0 && o1) {
            op.kind = (b0 & b1) ? SV_OP_NEG : SV_OP_NOP;
        } else if (o0 ? b0 : b1) {
            op.t[0] = o0 ? op.t[1] : op.t[0];
            op.kind = SV_OP_ZSIGN;
        } else {
            op.kind = SV_OP_NOP;
        }
    }
    return op;
}

__device__ __forceinline__ bool has_out_target(const DevOp &op) {
    return op.t[0] >= kOutTarget || (op.kind == SV_CZ && op.t[1] >= kOutTarget);
}

template <typename R>
__device__ void apply_op(Cx<R> *t, int k, const DevOp &op, const R *coef, const Cx<R> *mats, bool adj) {
    const uint32_t T = 1u << k;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    switch (op.kind) {
    case SV_RY: {
        const R c = coef[2 * op.gate];
        const R s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        const int b = op.t[0];
        for (uint32_t p = tid; p < T / 2; p += nt) {
            const uint32_t i0 = ins0(p, b), i1 = i0 | (1u << b);
            Cx<R> u = t[i0], v = t[i1];
            rot<R>(u, v, c, s);
            t[i0] = u;
            t[i1] = v;
        }
        break;
    }
    case SV_RZ: {
        // diag(e^{-i theta/2}, e^{+i theta/2})
        const R c = coef[2 * op.gate];
        const R s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        const int b = op.t[0];
        for (uint32_t p = tid; p < T; p += nt) {
            const R ss = ((p >> b) & 1u) ? s : -s;
            const Cx<R> v = t[p];
            t[p] = mk<R>(c * v.x - ss * v.y, c * v.y + ss * v.x);
        }
        break;
    }
    case SV_CZ: {
        const int a = min((int)op.t[0], (int)op.t[1]), b = max((int)op.t[0], (int)op.t[1]);
        const uint32_t both = (1u << a) | (1u << b);
        for (uint32_t p = tid; p < T / 4; p += nt) {
            const uint32_t i = ins0(ins0(p, a), b) | both;
            const Cx<R> v = t[i];
            t[i] = mk<R>(-v.x, -v.y);
        }
        break;
    }
    case SV_OP_PHASE: {
        const R c = coef[2 * op.gate];
        const R s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        const R ss = op.t[0] ? s : -s;
        for (uint32_t p = tid; p < T; p += nt) {
            const Cx<R> v = t[p];
            t[p] = mk<R>(c * v.x - ss * v.y, c * v.y + ss * v.x);
        }
        break;
    }
    case SV_OP_ZSIGN: {
        const int b = op.t[0];
        for (uint32_t p = tid; p < T / 2; p += nt) {
            const uint32_t i = ins0(p, b) | (1u << b);
            const Cx<R> v = t[i];
            t[i] = mk<R>(-v.x, -v.y);
        }
        break;
    }
    case SV_OP_NEG: {
        for (uint32_t p = tid; p < T; p += nt) t[p] = mk<R>(-t[p].x, -t[p].y);
        break;
    }
    case SV_GIVENS: {
        // span{|qa=1,qb=0>, |qa=0,qb=1>}
        const R c = coef[2 * op.gate];
        const R s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        const int qa = op.t[0], qb = op.t[1];
        const int lo = min(qa, qb), hi = max(qa, qb);
        for (uint32_t p = tid; p < T / 4; p += nt) {
            const uint32_t base = ins0(ins0(p, lo), hi);
            const uint32_t iu = base | (1u << qa), iv = base | (1u << qb);
            Cx<R> u = t[iu], v = t[iv];
            rot<R>(u, v, c, s);
            t[iu] = u;
            t[iv] = v;
        }
        break;
    }
    case SV_DEXC: {
        // span{|q0=q1=1, q2=q3=0>, |q2=q3=1, q0=q1=0>}
        const R c = coef[2 * op.gate];
        const R s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        int srt[4] = {op.t[0], op.t[1], op.t[2], op.t[3]};
        sort4(srt, 4);
        const uint32_t mu = (1u << op.t[0]) | (1u << op.t[1]);
        const uint32_t mv = (1u << op.t[2]) | (1u << op.t[3]);
        for (uint32_t p = tid; p < T / 16; p += nt) {
            uint32_t base = p;
            for (int i = 0; i < 4; ++i) base = ins0(base, srt[i]);
            Cx<R> u = t[base | mu], v = t[base | mv];
            rot<R>(u, v, c, s);
            t[base | mu] = u;
            t[base | mv] = v;
        }
        break;
    }
    case SV_MAT1:
    case SV_MAT2:
    case SV_MAT4:
        apply_dense_op<R>(t, k, op, mats, adj);
        break;
    default:
        break;
    }
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gradient part Im<lambda|G|psi> of one gate over the thread's index groups,
// then U^dagger on both tiles.  G = Y (RY), Z (RZ), Y on the two-state
// subspace (GIVENS, DEXC).  For a pair (u, v) with G u = i v, G v = -i u:
//   Im<lambda|G|psi> = Re(conj(lam_v) psi_u) - Re(conj(lam_u) psi_v).
template <typename R>
__device__ R adjoint_op(Cx<R> *tp, Cx<R> *tl, int k, const DevOp &op, const R *coef, const Cx<R> *mats) {
    const uint32_t T = 1u << k;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    R g = 0;
    switch (op.kind) {
    case SV_RY: {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        const int b = op.t[0];
        for (uint32_t p = tid; p < T / 2; p += nt) {
            const uint32_t i0 = ins0(p, b), i1 = i0 | (1u << b);
            Cx<R> pu = tp[i0], pv = tp[i1], lu = tl[i0], lv = tl[i1];
            g += (lv.x * pu.x + lv.y * pu.y) - (lu.x * pv.x + lu.y * pv.y);
            rot<R>(pu, pv, c, s);
            rot<R>(lu, lv, c, s);
            tp[i0] = pu; tp[i1] = pv; tl[i0] = lu; tl[i1] = lv;
        }
        break;
    }
    case SV_RZ: {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        const int b = op.t[0];
        for (uint32_t p = tid; p < T; p += nt) {
            const bool one = (p >> b) & 1u;
            const R ss = one ? s : -s;
            Cx<R> pv = tp[p], lv = tl[p];
            const R im = lv.x * pv.y - lv.y * pv.x;      // Im(conj(lam) psi)
            g += one ? -im : im;
            tp[p] = mk<R>(c * pv.x - ss * pv.y, c * pv.y + ss * pv.x);
            tl[p] = mk<R>(c * lv.x - ss * lv.y, c * lv.y + ss * lv.x);
        }
        break;
    }
    case SV_OP_PHASE: {
        // RZ on a qubit outside the tile: its bit is the same for every amplitude here
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        const bool one = op.t[0] != 0;
        const R ss = one ? s : -s;
        for (uint32_t p = tid; p < T; p += nt) {
            Cx<R> pv = tp[p], lv = tl[p];
            const R im = lv.x * pv.y - lv.y * pv.x;
            g += one ? -im : im;
            tp[p] = mk<R>(c * pv.x - ss * pv.y, c * pv.y + ss * pv.x);
            tl[p] = mk<R>(c * lv.x - ss * lv.y, c * lv.y + ss * lv.x);
        }
        break;
    }
    case SV_OP_ZSIGN:
    case SV_OP_NEG:
    case SV_OP_NOP:
        apply_op<R>(tp, k, op, coef, mats, true);
        apply_op<R>(tl, k, op, coef, mats, true);
        break;
    case SV_GIVENS: {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        const int qa = op.t[0], qb = op.t[1];
        const int lo = min(qa, qb), hi = max(qa, qb);
        for (uint32_t p = tid; p < T / 4; p += nt) {
            const uint32_t base = ins0(ins0(p, lo), hi);
            const uint32_t iu = base | (1u << qa), iv = base | (1u << qb);
            Cx<R> pu = tp[iu], pv = tp[iv], lu = tl[iu], lv = tl[iv];
            g += (lv.x * pu.x + lv.y * pu.y) - (lu.x * pv.x + lu.y * pv.y);
            rot<R>(pu, pv, c, s);
            rot<R>(lu, lv, c, s);
            tp[iu] = pu; tp[iv] = pv; tl[iu] = lu; tl[iv] = lv;
        }
        break;
    }
    case SV_DEXC: {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        int srt[4] = {op.t[0], op.t[1], op.t[2], op.t[3]};
        sort4(srt, 4);
        const uint32_t mu = (1u << op.t[0]) | (1u << op.t[1]);
        const uint32_t mv = (1u << op.t[2]) | (1u << op.t[3]);
        for (uint32_t p = tid; p < T / 16; p += nt) {
            uint32_t base = p;
            for (int i = 0; i < 4; ++i) base = ins0(base, srt[i]);
            const uint32_t iu = base | mu, iv = base | mv;
            Cx<R> pu = tp[iu], pv = tp[iv], lu = tl[iu], lv = tl[iv];
            g += (lv.x * pu.x + lv.y * pu.y) - (lu.x * pv.x + lu.y * pv.y);
            rot<R>(pu, pv, c, s);
            rot<R>(lu, lv, c, s);
            tp[iu] = pu; tp[iv] = pv; tl[iu] = lu; tl[iv] = lv;
        }
        break;
    }
    default:
        apply_op<R>(tp, k, op, coef, mats, true);
        apply_op<R>(tl, k, op, coef, mats, true);
        break;
    }
    return g;
}

__device__ __forceinline__ bool has_param(int kind) {
    return kind == SV_RY || kind == SV_RZ || kind == SV_GIVENS || kind == SV_DEXC || kind == SV_OP_PHASE;
}

// ------------------------------------------------------------------ K-GATE --
template <typename R>
__global__ void __launch_bounds__(512) k_gate_pass(Cx<R> *__restrict__ psi, const GatePassArgs a,
                                                   const DevOp *__restrict__ ops, const R *__restrict__ coef,
                                                   const Cx<R> *__restrict__ mats) {
    extern __shared__ __align__(16) unsigned char smem[];
    Cx<R> *tile = reinterpret_cast<Cx<R> *>(smem);
    const uint32_t T = 1u << a.k;
    const uint32_t nh = 1u << (a.k - a.nlow);
    uint64_t *hioff = reinterpret_cast<uint64_t *>(tile + T);
    for (uint32_t j = threadIdx.x; j < nh; j += blockDim.x) hioff[j] = deposit(j, a.hi, a.nhi);
    __syncthreads();
    const uint64_t ntiles = 1ull << a.nout;
    const uint32_t lowmask = (1u << a.nlow) - 1u;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const uint64_t base = deposit(ti, a.out, a.nout);
        for (uint32_t j = threadIdx.x; j < T; j += blockDim.x)
            tile[j] = psi[base | hioff[j >> a.nlow] | (j & lowmask)];
        __syncthreads();
        for (int o = a.op_begin; o < a.op_end; ++o) {
            const DevOp op = resolve_out(ops[o], base);
            apply_op<R>(tile, a.k, op, coef, mats, false);
            __syncthreads();
        }
        for (uint32_t j = threadIdx.x; j < T; j += blockDim.x)
            psi[base | hioff[j >> a.nlow] | (j & lowmask)] = tile[j];
        __syncthreads();
    }
}

// ------------------------------------------------------------------- K-ADJ --
template <typename R>
__global__ void __launch_bounds__(512) k_adj_pass(Cx<R> *__restrict__ psi, Cx<R> *__restrict__ lam,
                                                  const GatePassArgs a, const DevOp *__restrict__ ops,
                                                  const R *__restrict__ coef, const Cx<R> *__restrict__ mats,
                                                  double *__restrict__ part, int part_stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t T = 1u << a.k;
    const uint32_t nh = 1u << (a.k - a.nlow);
    const int nops = a.op_end - a.op_begin;
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Cx<R> *tp = reinterpret_cast<Cx<R> *>(smem);
    Cx<R> *tl = tp + T;
    uint64_t *hioff = reinterpret_cast<uint64_t *>(tl + T);
    double *acc = reinterpret_cast<double *>(hioff + nh);
    for (uint32_t j = threadIdx.x; j < nh; j += blockDim.x) hioff[j] = deposit(j, a.hi, a.nhi);
    for (int j = threadIdx.x; j < nops * nwarps; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    const uint64_t ntiles = 1ull << a.nout;
    const uint32_t lowmask = (1u << a.nlow) - 1u;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const uint64_t base = deposit(ti, a.out, a.nout);
        for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) {
            const uint64_t gi = base | hioff[j >> a.nlow] | (j & lowmask);
            tp[j] = psi[gi];
            tl[j] = lam[gi];
        }
        __syncthreads();
        for (int o = a.op_end - 1; o >= a.op_begin; --o) {
            const DevOp op = resolve_out(ops[o], base);
            R g = adjoint_op<R>(tp, tl, a.k, op, coef, mats);
            if (has_param(op.kind)) {
                g = warp_sum<R>(g);
                if (lane == 0) acc[(o - a.op_begin) * nwarps + warp] += (double)g;
            }
            __syncthreads();
        }
        for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) {
            const uint64_t gi = base | hioff[j >> a.nlow] | (j & lowmask);
            psi[gi] = tp[j];
            lam[gi] = tl[j];
        }
        __syncthreads();
    }
    for (int o = threadIdx.x; o < nops; o += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += acc[o * nwarps + w];
        part[(size_t)blockIdx.x * part_stride + a.op_begin + o] = s;
    }
}

// ---------------------------------------------------------- cp.async --
// 16-byte asynchronous global -> shared copies with commit / wait groups.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Complex load from a 32-bit shared-window address (the coset loops compute
// partner addresses as shared offsets, so no 64-bit pointer arithmetic).
// Ordered against the barriers around it by being volatile.
template <typename R> __device__ __forceinline__ Cx<R> lds_cx(uint32_t addr);
template <> __device__ __forceinline__ Cx<float> lds_cx<float>(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}
template <> __device__ __forceinline__ Cx<double> lds_cx<double>(uint32_t addr) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr));
    return v;
}
// The same for complex64 at addr + OFF (OFF a compile-time byte offset, so
// the address is one register plus an immediate).
template <int OFF> __device__ __forceinline__ float2 lds_f2_off(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF));
    return v;
}

// ------------------------------------------------- register-blocked passes --
// A pass of RY / RZ / CZ / 1-qubit matrices runs in phases (host planned):
// in a phase each of the 512 threads holds the 2^RB amplitudes spanned by
// the phase's register bits (rmask) of the staged tile, gathered from shared
// memory; non-diagonal gates act on register bits, diagonal gates on any bit
// (a thread bit just selects the phase or sign for all of its registers).
// One shared-memory transpose per phase instead of one barrier per gate.
__device__ __forceinline__ uint32_t swz_tile(uint32_t i) {
    return swz_slot(i);   // bijection; spreads strided lanes over the banks
}

template <typename R, int V, int B>
__device__ __forceinline__ void reg_rot(Cx<R> *x, R c, R s) {
    if constexpr (sizeof(R) == 4) {
        const RotPairs k = rot_pairs(c, s);   // once per gate, not per pair
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (!(v & (1 << B))) rot_packed(x[v], x[v | (1 << B)], k);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (!(v & (1 << B))) rot<R>(x[v], x[v | (1 << B)], c, s);
    }
}
template <typename R, int V, int B>
__device__ __forceinline__ void reg_mat1(Cx<R> *x, const Cx<R> *M, bool adj) {
    const Cx<R> m00 = mel<R>(M, 2, 0, 0, adj), m01 = mel<R>(M, 2, 0, 1, adj);
    const Cx<R> m10 = mel<R>(M, 2, 1, 0, adj), m11 = mel<R>(M, 2, 1, 1, adj);
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (!(v & (1 << B))) {
            const Cx<R> a = x[v], b = x[v | (1 << B)];
            x[v] = mk<R>(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                         m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x);
            x[v | (1 << B)] = mk<R>(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                                    m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x);
        }
}
// multiply by (c, s) where bit B of v is 1 and by (c, -s) where it is 0
template <typename R, int V, int B>
__device__ __forceinline__ void reg_rz(Cx<R> *x, R c, R s) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const R ss = (v & (1 << B)) ? s : -s;
        x[v] = mk<R>(c * x[v].x - ss * x[v].y, c * x[v].y + ss * x[v].x);
    }
}
template <typename R, int V, int B0, int B1>
__device__ __forceinline__ void reg_cz2(Cx<R> *x) {
#pragma unroll
    for (int v = 0; v < V; ++v)
        if ((v & (1 << B0)) && (v & (1 << B1))) x[v] = mk<R>(-x[v].x, -x[v].y);
}
template <typename R, int V, int B>
__device__ __forceinline__ void reg_neg_bit(Cx<R> *x) {
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (v & (1 << B)) x[v] = mk<R>(-x[v].x, -x[v].y);
}

#define SV_REG_SWITCH(b, CALL)                                   \
    switch (b) {                                                 \
    case 0: CALL(0); break;                                      \
    case 1: if constexpr (RB > 1) { CALL(1); } break;            \
    case 2: if constexpr (RB > 2) { CALL(2); } break;            \
    case 3: if constexpr (RB > 3) { CALL(3); } break;            \
    case 4: if constexpr (RB > 4) { CALL(4); } break;            \
    default: break;                                              \
    }

// One gate on the registers of a phase.  rmask: register tile bits; base:
// the thread's tile index bits outside rmask.
template <typename R, int RB>
__device__ __forceinline__ void reg_apply(Cx<R> *x, const DevOp &op, uint32_t rmask, uint32_t base, const R *coef,
                                          const Cx<R> *mats, bool adj) {
    constexpr int V = 1 << RB;
    const int t0 = op.t[0];
    const int b0 = __popc(rmask & ((1u << t0) - 1u));
    switch (op.kind) {
    case SV_RY: {
        const R c = coef[2 * op.gate], s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
#define SV_C(B) reg_rot<R, V, B>(x, c, s)
        SV_REG_SWITCH(b0, SV_C)
#undef SV_C
        break;
    }
    case SV_MAT1: {
        const Cx<R> *M = mats + op.mat;
#define SV_C(B) reg_mat1<R, V, B>(x, M, adj)
        SV_REG_SWITCH(b0, SV_C)
#undef SV_C
        break;
    }
    case SV_RZ: {
        const R c = coef[2 * op.gate], s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        if ((rmask >> t0) & 1u) {
#define SV_C(B) reg_rz<R, V, B>(x, c, s)
            SV_REG_SWITCH(b0, SV_C)
#undef SV_C
        } else {
            const R ss = ((base >> t0) & 1u) ? s : -s;
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = mk<R>(c * x[v].x - ss * x[v].y, c * x[v].y + ss * x[v].x);
        }
        break;
    }
    case SV_CZ: {
        const int t1 = op.t[1];
        const bool r0 = (rmask >> t0) & 1u, r1 = (rmask >> t1) & 1u;
        if (r0 && r1) {
            const int b1 = __popc(rmask & ((1u << t1) - 1u));
            const int lo = min(b0, b1), hi = max(b0, b1);
            switch (lo * 8 + hi) {
#define SV_CZ_CASE(L, H) case L * 8 + H: if constexpr (RB > H) { reg_cz2<R, V, L, H>(x); } break;
                SV_CZ_CASE(0, 1) SV_CZ_CASE(0, 2) SV_CZ_CASE(0, 3) SV_CZ_CASE(0, 4)
                SV_CZ_CASE(1, 2) SV_CZ_CASE(1, 3) SV_CZ_CASE(1, 4)
                SV_CZ_CASE(2, 3) SV_CZ_CASE(2, 4) SV_CZ_CASE(3, 4)
#undef SV_CZ_CASE
            default: break;
            }
        } else if (r0 || r1) {
            const int tr = r0 ? t0 : t1, tt = r0 ? t1 : t0;
            if ((base >> tt) & 1u) {
                const int br = __popc(rmask & ((1u << tr) - 1u));
#define SV_C(B) reg_neg_bit<R, V, B>(x)
                SV_REG_SWITCH(br, SV_C)
#undef SV_C
            }
        } else if (((base >> t0) & (base >> t1)) & 1u) {
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = mk<R>(-x[v].x, -x[v].y);
        }
        break;
    }
    case SV_OP_PHASE: {
        const R c = coef[2 * op.gate], s = adj ? -coef[2 * op.gate + 1] : coef[2 * op.gate + 1];
        const R ss = op.t[0] ? s : -s;
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = mk<R>(c * x[v].x - ss * x[v].y, c * x[v].y + ss * x[v].x);
        break;
    }
    case SV_OP_ZSIGN: {
        if ((rmask >> t0) & 1u) {
#define SV_C(B) reg_neg_bit<R, V, B>(x)
            SV_REG_SWITCH(b0, SV_C)
#undef SV_C
        } else if ((base >> t0) & 1u) {
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = mk<R>(-x[v].x, -x[v].y);
        }
        break;
    }
    case SV_OP_NEG: {
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = mk<R>(-x[v].x, -x[v].y);
        break;
    }
    default:
        break;
    }
}

// Gradient part Im<lambda|G|psi> of a parametric gate on the registers (G = Y
// for RY, Z for RZ), then U^dagger on both register sets.
template <typename R, int V, int B>
__device__ __forceinline__ R reg_ry_adj(Cx<R> *p, Cx<R> *l, R c, R s) {
    R g = 0;
    if constexpr (sizeof(R) == 4) {
        const RotPairs k = rot_pairs(c, s);
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (!(v & (1 << B))) {
                const int w = v | (1 << B);
                g += (l[w].x * p[v].x + l[w].y * p[v].y) - (l[v].x * p[w].x + l[v].y * p[w].y);
                rot_packed(p[v], p[w], k);
                rot_packed(l[v], l[w], k);
            }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (!(v & (1 << B))) {
                const int w = v | (1 << B);
                g += (l[w].x * p[v].x + l[w].y * p[v].y) - (l[v].x * p[w].x + l[v].y * p[w].y);
                rot<R>(p[v], p[w], c, s);
                rot<R>(l[v], l[w], c, s);
            }
    }
    return g;
}
template <typename R, int V, int B>
__device__ __forceinline__ R reg_rz_adj(Cx<R> *p, Cx<R> *l, R c, R s) {
    R g = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const bool one = v & (1 << B);
        const R im = l[v].x * p[v].y - l[v].y * p[v].x;
        g += one ? -im : im;
        const R ss = one ? s : -s;
        p[v] = mk<R>(c * p[v].x - ss * p[v].y, c * p[v].y + ss * p[v].x);
        l[v] = mk<R>(c * l[v].x - ss * l[v].y, c * l[v].y + ss * l[v].x);
    }
    return g;
}

template <typename R, int RB>
__device__ __forceinline__ R reg_adjoint(Cx<R> *p, Cx<R> *l, const DevOp &op, uint32_t rmask, uint32_t base,
                                         const R *coef, const Cx<R> *mats) {
    constexpr int V = 1 << RB;
    const int t0 = op.t[0];
    const int b0 = __popc(rmask & ((1u << t0) - 1u));
    R g = 0;
    if (op.kind == SV_RY) {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
#define SV_C(B) g = reg_ry_adj<R, V, B>(p, l, c, s)
        SV_REG_SWITCH(b0, SV_C)
#undef SV_C
    } else if (op.kind == SV_RZ || op.kind == SV_OP_PHASE) {
        const R c = coef[2 * op.gate], s = -coef[2 * op.gate + 1];
        if (op.kind == SV_RZ && ((rmask >> t0) & 1u)) {
#define SV_C(B) g = reg_rz_adj<R, V, B>(p, l, c, s)
            SV_REG_SWITCH(b0, SV_C)
#undef SV_C
        } else {
            // the bit is the same for all registers: a thread bit, or a qubit outside the tile
            const bool one = op.kind == SV_OP_PHASE ? op.t[0] != 0 : ((base >> t0) & 1u) != 0;
            const R ss = one ? s : -s;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const R im = l[v].x * p[v].y - l[v].y * p[v].x;
                g += one ? -im : im;
                p[v] = mk<R>(c * p[v].x - ss * p[v].y, c * p[v].y + ss * p[v].x);
                l[v] = mk<R>(c * l[v].x - ss * l[v].y, c * l[v].y + ss * l[v].x);
            }
        }
    } else {
        reg_apply<R, RB>(p, op, rmask, base, coef, mats, true);
        reg_apply<R, RB>(l, op, rmask, base, coef, mats, true);
    }
    return g;
}
#undef SV_REG_SWITCH

// Thread's tile index bits outside rmask, and the register spread table.
template <int RB>
__device__ __forceinline__ void phase_index(uint32_t rmask, int k, uint32_t &base, uint32_t *sp) {
    const uint32_t tb = ((k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u)) & ~rmask;
    base = 0;
    uint32_t t = threadIdx.x, m = tb;
    while (m) {
        const uint32_t lowbit = m & (0u - m);
        if (t & 1u) base |= lowbit;
        t >>= 1;
        m ^= lowbit;
    }
    uint32_t rb[RB];
    uint32_t rm = rmask;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
        rb[i] = rm & (0u - rm);
        rm ^= rb[i];
    }
    sp[0] = 0;
#pragma unroll
    for (int v = 1; v < (1 << RB); ++v) sp[v] = sp[v & (v - 1)] | rb[__ffs(v) - 1];
}

// The thread's tile bits outside rmask when the lane bits of the thread
// index hold the tile bits in `lanes` (ascending) and the other thread index
// bits hold the remaining non-register bits (ascending).
__device__ __forceinline__ uint32_t phase_base(uint32_t rmask, uint32_t lanes, int k) {
    const uint32_t all = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u);
    uint32_t base = 0, t = threadIdx.x;
    for (uint32_t m = lanes; m; m &= m - 1, t >>= 1)
        if (t & 1u) base |= m & (0u - m);
    for (uint32_t m = all & ~rmask & ~lanes; m; m &= m - 1, t >>= 1)
        if (t & 1u) base |= m & (0u - m);
    return base;
}

// ---- register-blocked pass execution ----------------------------------
// Complex64 amplitudes stay in one 64-bit register pair (re, im) while a
// phase is in registers, so that rotations with real coefficients are pure
// packed f32x2 arithmetic; complex128 ones are double2.
template <typename R> struct RegT;
template <> struct RegT<float> { using T = unsigned long long; };
template <> struct RegT<double> { using T = double2; };
template <typename R> using RA = typename RegT<R>::T;

template <typename R> __device__ __forceinline__ Cx<R> ra_cx(RA<R> a);
template <> __device__ __forceinline__ float2 ra_cx<float>(unsigned long long a) { return f2_unpack(a); }
template <> __device__ __forceinline__ double2 ra_cx<double>(double2 a) { return a; }
template <typename R> __device__ __forceinline__ RA<R> cx_ra(Cx<R> a);
template <> __device__ __forceinline__ unsigned long long cx_ra<float>(float2 a) { return f2_pack(a.x, a.y); }
template <> __device__ __forceinline__ double2 cx_ra<double>(double2 a) { return a; }

template <typename R> __device__ __forceinline__ RA<R> ra_neg(RA<R> a);
template <> __device__ __forceinline__ unsigned long long ra_neg<float>(unsigned long long a) {
    return a ^ 0x8000000080000000ull;
}
template <> __device__ __forceinline__ double2 ra_neg<double>(double2 a) { return make_double2(-a.x, -a.y); }

// a * w (complex), or a * conj(w)
template <typename R>
__device__ __forceinline__ RA<R> ra_cmul(RA<R> a, Cx<R> w) {
    const Cx<R> x = ra_cx<R>(a);
    return cx_ra<R>(mk<R>(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x));
}

// One RY's coefficients, packed once per gate.
template <typename R> struct RotK;
template <> struct RotK<float> { unsigned long long C, S, NS; };
template <> struct RotK<double> { double c, s; };
template <typename R> __device__ __forceinline__ RotK<R> rotk(R c, R s);
template <> __device__ __forceinline__ RotK<float> rotk<float>(float c, float s) {
    return {f2_pack(c, c), f2_pack(s, s), f2_pack(-s, -s)};
}
template <> __device__ __forceinline__ RotK<double> rotk<double>(double c, double s) { return {c, s}; }

// (u, v) <- (c u - s v, s u + c v) on every pair of register bit B
template <typename R, int V, int B>
__device__ __forceinline__ void ra_rot(RA<R> *x, const RotK<R> &k) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if (v & (1 << B)) continue;
        const int w = v | (1 << B);
        if constexpr (sizeof(R) == 4) {
            unsigned long long t, uu, vv;
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x[w]), "l"(k.NS));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(uu) : "l"(x[v]), "l"(k.C), "l"(t));
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x[w]), "l"(k.C));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(vv) : "l"(x[v]), "l"(k.S), "l"(t));
            x[v] = uu;
            x[w] = vv;
        } else {
            const double2 a = x[v], b = x[w];
            x[v] = make_double2(k.c * a.x - k.s * b.x, k.c * a.y - k.s * b.y);
            x[w] = make_double2(k.s * a.x + k.c * b.x, k.s * a.y + k.c * b.y);
        }
    }
}

// RY with its larger coefficient factored out (the factor is common to every
// amplitude of the tile, so a pass carries the product of the factors and
// applies it once when the tile is stored):
//   |c| >= |s|: RY = c [[1, -t], [t, 1]], t = s / c   (form A)
//   |c| <  |s|: RY = s [[t, -1], [1, t]], t = c / s   (form B)
// so |t| <= 1, the factor is at least 1/sqrt(2) in magnitude, and a pair
// costs two fused multiply-adds (form B: plus a sign flip) instead of two
// products and two fused multiply-adds.
template <typename R> struct RotF;
template <> struct RotF<float> { unsigned long long T, NT; };
template <> struct RotF<double> { double t; };
template <typename R> __device__ __forceinline__ RotF<R> rotf(R t);
template <> __device__ __forceinline__ RotF<float> rotf<float>(float t) { return {f2_pack(t, t), f2_pack(-t, -t)}; }
template <> __device__ __forceinline__ RotF<double> rotf<double>(double t) { return {t}; }

// factored form (t, factor) and form bit of an RY with coefficients (c, s)
template <typename R> __device__ __forceinline__ Cx<R> ry_factored(R c, R s, int &form_b) {
    const bool b = fabs(s) > fabs(c);
    form_b = b ? 1 : 0;
    return b ? mk<R>(c / s, s) : mk<R>(s / c, c);
}

template <typename R, int V, int B, bool FB>
__device__ __forceinline__ void ra_rotf(RA<R> *x, const RotF<R> &k) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if (v & (1 << B)) continue;
        const int w = v | (1 << B);
        if constexpr (sizeof(R) == 4) {
            unsigned long long uu, vv;
            if (FB) {   // (t u - v, u + t v)
                const unsigned long long nw = x[w] ^ 0x8000000080000000ull;
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(uu) : "l"(x[v]), "l"(k.T), "l"(nw));
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(vv) : "l"(x[w]), "l"(k.T), "l"(x[v]));
            } else {    // (u - t v, v + t u)
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(uu) : "l"(x[w]), "l"(k.NT), "l"(x[v]));
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(vv) : "l"(x[v]), "l"(k.T), "l"(x[w]));
            }
            x[v] = uu;
            x[w] = vv;
        } else {
            const double2 a = x[v], b = x[w];
            if (FB) {
                x[v] = make_double2(fma(k.t, a.x, -b.x), fma(k.t, a.y, -b.y));
                x[w] = make_double2(fma(k.t, b.x, a.x), fma(k.t, b.y, a.y));
            } else {
                x[v] = make_double2(fma(-k.t, b.x, a.x), fma(-k.t, b.y, a.y));
                x[w] = make_double2(fma(k.t, a.x, b.x), fma(k.t, a.y, b.y));
            }
        }
    }
}

// one factored RY on register bit b (0..RB-1) in form fb
template <typename R, int V, int RB>
__device__ __forceinline__ void ra_rotf_bit(RA<R> *x, int b, bool fb, const RotF<R> &k) {
    switch (b * 2 + (fb ? 1 : 0)) {
    case 0: ra_rotf<R, V, 0, false>(x, k); break;
    case 1: ra_rotf<R, V, 0, true>(x, k); break;
    case 2: if constexpr (RB > 1) ra_rotf<R, V, 1, false>(x, k); break;
    case 3: if constexpr (RB > 1) ra_rotf<R, V, 1, true>(x, k); break;
    case 4: if constexpr (RB > 2) ra_rotf<R, V, 2, false>(x, k); break;
    case 5: if constexpr (RB > 2) ra_rotf<R, V, 2, true>(x, k); break;
    case 6: if constexpr (RB > 3) ra_rotf<R, V, 3, false>(x, k); break;
    case 7: if constexpr (RB > 3) ra_rotf<R, V, 3, true>(x, k); break;
    default: break;
    }
}

// Gradient part of an RY on register bit B: sum over pairs (v, w = v | bit B)
// of Re(conj(l_w) p_v) - Re(conj(l_v) p_w)  (= Im<lambda|Y|psi> on the pairs).
template <typename R, int V, int B>
__device__ __forceinline__ R ra_ry_grad(const RA<R> *p, const RA<R> *l) {
    if constexpr (sizeof(R) == 4) {
        unsigned long long P = 0, M = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (v & (1 << B)) continue;
            const int w = v | (1 << B);
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(P) : "l"(l[w]), "l"(p[v]), "l"(P));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(M) : "l"(l[v]), "l"(p[w]), "l"(M));
        }
        const float2 a = f2_unpack(P), b = f2_unpack(M);
        return (a.x + a.y) - (b.x + b.y);
    } else {
        double g = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (v & (1 << B)) continue;
            const int w = v | (1 << B);
            g += (l[w].x * p[v].x + l[w].y * p[v].y) - (l[v].x * p[w].x + l[v].y * p[w].y);
        }
        return g;
    }
}

// sb[b] = sum_v (-1)^{bit b of v} tv[v] for every register bit b, by
// halving: pair sums feed the next bit, pair differences sum into sb[b].
template <typename R, int RB>
__device__ __forceinline__ void signed_bit_sums(const R *tv, R *sb) {
    constexpr int V = 1 << RB;
    R cur[V];
#pragma unroll
    for (int v = 0; v < V; ++v) cur[v] = tv[v];
#pragma unroll
    for (int b = 0, n = V; b < RB; ++b, n >>= 1) {
        R d = 0;
#pragma unroll
        for (int k = 0; k < n / 2; ++k) {
            d += cur[2 * k] - cur[2 * k + 1];
            cur[k] = cur[2 * k] + cur[2 * k + 1];
        }
        sb[b] = d;
    }
}

// Rotation (u, v) <- (c u - s v, s u + c v) of every register pair (u = x[v]
// with (v & (MU | MV)) == MU, v' = v ^ MU ^ MV): RY on bit B is MU = 0,
// MV = 1 << B; a Givens rotation MU = 1 << a, MV = 1 << b; the double
// excitation MU, MV = the two bit pairs.
template <typename R, int V, int MU, int MV>
__device__ __forceinline__ void ra_pair_rot(RA<R> *x, const RotK<R> &k) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if ((v & (MU | MV)) != MU) continue;
        const int w = v ^ MU ^ MV;
        if constexpr (sizeof(R) == 4) {
            unsigned long long t, uu, vv;
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x[w]), "l"(k.NS));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(uu) : "l"(x[v]), "l"(k.C), "l"(t));
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x[w]), "l"(k.C));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(vv) : "l"(x[v]), "l"(k.S), "l"(t));
            x[v] = uu;
            x[w] = vv;
        } else {
            const double2 a = x[v], b = x[w];
            x[v] = make_double2(k.c * a.x - k.s * b.x, k.c * a.y - k.s * b.y);
            x[w] = make_double2(k.s * a.x + k.c * b.x, k.s * a.y + k.c * b.y);
        }
    }
}
// Gradient part Im<lambda|G|psi> of such a rotation (G the subspace Y):
// sum over the pairs of Re(conj(l_v') p_v) - Re(conj(l_v) p_v').
template <typename R, int V, int MU, int MV>
__device__ __forceinline__ R ra_pair_grad(const RA<R> *p, const RA<R> *l) {
    R g = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if ((v & (MU | MV)) != MU) continue;
        const int w = v ^ MU ^ MV;
        const Cx<R> pv = ra_cx<R>(p[v]), pw = ra_cx<R>(p[w]), lv = ra_cx<R>(l[v]), lw = ra_cx<R>(l[w]);
        g += (lw.x * pv.x + lw.y * pv.y) - (lv.x * pw.x + lv.y * pw.y);
    }
    return g;
}

// Givens rotation on register bits (A, B), A holding the "1" of u; and the
// double excitation on the four register bits with u's pair MU.
#define SV_GIVENS_SWITCH(ra, rb, CALL)                                                       \
    switch ((ra) * 4 + (rb)) {                                                               \
    case 1: CALL(1, 2); break;   case 2: if constexpr (RB > 2) { CALL(1, 4); } break;        \
    case 3: if constexpr (RB > 3) { CALL(1, 8); } break;                                     \
    case 4: CALL(2, 1); break;   case 6: if constexpr (RB > 2) { CALL(2, 4); } break;        \
    case 7: if constexpr (RB > 3) { CALL(2, 8); } break;                                     \
    case 8: if constexpr (RB > 2) { CALL(4, 1); } break;                                     \
    case 9: if constexpr (RB > 2) { CALL(4, 2); } break;                                     \
    case 11: if constexpr (RB > 3) { CALL(4, 8); } break;                                    \
    case 12: if constexpr (RB > 3) { CALL(8, 1); } break;                                    \
    case 13: if constexpr (RB > 3) { CALL(8, 2); } break;                                    \
    case 14: if constexpr (RB > 3) { CALL(8, 4); } break;                                    \
    default: break;                                                                          \
    }
#define SV_DEXC_SWITCH(mu, CALL)                                                             \
    if constexpr (RB == 4) {                                                                 \
        switch (mu) {                                                                        \
        case 3: CALL(3, 12); break;  case 5: CALL(5, 10); break;  case 6: CALL(6, 9); break; \
        case 9: CALL(9, 6); break;   case 10: CALL(10, 5); break; case 12: CALL(12, 3); break; \
        default: break;                                                                      \
        }                                                                                    \
    }

// Four values reduced over a warp at once: lane L ends with the warp total
// of value L >> 3 (6 shuffles instead of 20).
template <typename R>
__device__ __forceinline__ R warp_sum4(R v0, R v1, R v2, R v3) {
    const unsigned lane = threadIdx.x & 31u;
    const bool hi = lane & 16u;
    R k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
    k0 += __shfl_xor_sync(0xffffffffu, hi ? v0 : v2, 16);
    k1 += __shfl_xor_sync(0xffffffffu, hi ? v1 : v3, 16);
    const bool h8 = lane & 8u;
    R k = (h8 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

template <typename R, int V, int B>
__device__ __forceinline__ void ra_mat1(RA<R> *x, const Cx<R> *M, bool adj) {
    const Cx<R> m00 = mel<R>(M, 2, 0, 0, adj), m01 = mel<R>(M, 2, 0, 1, adj);
    const Cx<R> m10 = mel<R>(M, 2, 1, 0, adj), m11 = mel<R>(M, 2, 1, 1, adj);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if (v & (1 << B)) continue;
        const int w = v | (1 << B);
        const Cx<R> a = ra_cx<R>(x[v]), b = ra_cx<R>(x[w]);
        x[v] = cx_ra<R>(mk<R>(m00.x * a.x - m00.y * a.y + m01.x * b.x - m01.y * b.y,
                              m00.x * a.y + m00.y * a.x + m01.x * b.y + m01.y * b.x));
        x[w] = cx_ra<R>(mk<R>(m10.x * a.x - m10.y * a.y + m11.x * b.x - m11.y * b.y,
                              m10.x * a.y + m10.y * a.x + m11.x * b.y + m11.y * b.x));
    }
}

#define SV_RB_SWITCH(b, CALL)                                    \
    switch (b) {                                                 \
    case 0: CALL(0); break;                                      \
    case 1: if constexpr (RB > 1) { CALL(1); } break;            \
    case 2: if constexpr (RB > 2) { CALL(2); } break;            \
    case 3: if constexpr (RB > 3) { CALL(3); } break;            \
    default: break;                                              \
    }

// One operation applied by the generic path (OP steps) on register
// amplitudes: base = the thread's tile bits outside rmask; cs = (cos, sin)
// of the half angle (sin already negated for an inverse).
template <typename R, int RB>
__device__ void ra_apply_op(RA<R> *x, DevOp op, uint32_t rmask, uint32_t base, Cx<R> cs, const Cx<R> *mats,
                            bool adj) {
    constexpr int V = 1 << RB;
    const int t0 = op.t[0];
    const int b0 = __popc(rmask & ((1u << (t0 & 31)) - 1u));
    switch (op.kind) {
    case SV_RY: {
        const RotK<R> k = rotk<R>(cs.x, cs.y);
#define SV_C(B) ra_rot<R, V, B>(x, k)
        SV_RB_SWITCH(b0, SV_C)
#undef SV_C
        break;
    }
    case SV_MAT1: {
        const Cx<R> *M = mats + op.mat;
#define SV_C(B) ra_mat1<R, V, B>(x, M, adj)
        SV_RB_SWITCH(b0, SV_C)
#undef SV_C
        break;
    }
    case SV_GIVENS: {
        const RotK<R> k = rotk<R>(cs.x, cs.y);
        const int b1 = __popc(rmask & ((1u << op.t[1]) - 1u));
#define SV_C(MU, MV) ra_pair_rot<R, V, MU, MV>(x, k)
        SV_GIVENS_SWITCH(b0, b1, SV_C)
#undef SV_C
        break;
    }
    case SV_DEXC: {
        const RotK<R> k = rotk<R>(cs.x, cs.y);
        const int mu = (1 << b0) | (1 << __popc(rmask & ((1u << op.t[1]) - 1u)));
#define SV_C(MU, MV) ra_pair_rot<R, V, MU, MV>(x, k)
        SV_DEXC_SWITCH(mu, SV_C)
#undef SV_C
        break;
    }
    case SV_RZ: {
        if ((rmask >> t0) & 1u) {
            const Cx<R> w0 = mk<R>(cs.x, -cs.y), w1 = mk<R>(cs.x, cs.y);
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = ra_cmul<R>(x[v], ((v >> b0) & 1) ? w1 : w0);
        } else {
            const Cx<R> w = mk<R>(cs.x, ((base >> t0) & 1u) ? cs.y : -cs.y);
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = ra_cmul<R>(x[v], w);
        }
        break;
    }
    case SV_CZ: {
        const int t1 = op.t[1];
        const bool r0 = (rmask >> t0) & 1u, r1 = (rmask >> t1) & 1u;
        uint32_t negmask = 0;   // register amplitudes that change sign
        if (r0 && r1) {
            const int b1 = __popc(rmask & ((1u << t1) - 1u));
#pragma unroll
            for (int v = 0; v < V; ++v)
                if ((v >> b0) & (v >> b1) & 1) negmask |= 1u << v;
        } else if (r0 || r1) {
            const int tr = r0 ? t0 : t1, tt = r0 ? t1 : t0;
            if ((base >> tt) & 1u) {
                const int br = __popc(rmask & ((1u << tr) - 1u));
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if ((v >> br) & 1) negmask |= 1u << v;
            }
        } else if (((base >> t0) & (base >> t1)) & 1u) {
            negmask = 0xFFFFFFFFu;
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
            if ((negmask >> v) & 1u) x[v] = ra_neg<R>(x[v]);
        break;
    }
    case SV_OP_PHASE: {
        const Cx<R> w = mk<R>(cs.x, op.t[0] ? cs.y : -cs.y);
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = ra_cmul<R>(x[v], w);
        break;
    }
    case SV_OP_ZSIGN: {
        const bool reg = (rmask >> t0) & 1u;
        const bool thr = !reg && ((base >> t0) & 1u);
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (reg ? ((v >> b0) & 1) : thr) x[v] = ra_neg<R>(x[v]);
        break;
    }
    case SV_OP_NEG: {
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = ra_neg<R>(x[v]);
        break;
    }
    default:
        break;
    }
}

// Im(conj(l) p) per register amplitude
template <typename R>
__device__ __forceinline__ R ra_imdot(RA<R> l, RA<R> p) {
    const Cx<R> a = ra_cx<R>(l), b = ra_cx<R>(p);
    return a.x * b.y - a.y * b.x;
}

// Adjoint of one OP step: gradient part Im<lambda|G|psi> (RY: Y, RZ: Z), then
// U^dagger on both register sets.  cs holds (cos, -sin).
template <typename R, int RB>
__device__ R ra_adjoint_op(RA<R> *p, RA<R> *l, DevOp op, uint32_t rmask, uint32_t base, Cx<R> cs,
                           const Cx<R> *mats) {
    constexpr int V = 1 << RB;
    const int t0 = op.t[0];
    const int b0 = __popc(rmask & ((1u << (t0 & 31)) - 1u));
    R g = 0;
    if (op.kind == SV_RY) {
#define SV_C(B) g = ra_ry_grad<R, V, B>(p, l)
        SV_RB_SWITCH(b0, SV_C)
#undef SV_C
    } else if (op.kind == SV_GIVENS) {
        const int b1 = __popc(rmask & ((1u << op.t[1]) - 1u));
#define SV_C(MU, MV) g = ra_pair_grad<R, V, MU, MV>(p, l)
        SV_GIVENS_SWITCH(b0, b1, SV_C)
#undef SV_C
    } else if (op.kind == SV_DEXC) {
        const int mu = (1 << b0) | (1 << __popc(rmask & ((1u << op.t[1]) - 1u)));
#define SV_C(MU, MV) g = ra_pair_grad<R, V, MU, MV>(p, l)
        SV_DEXC_SWITCH(mu, SV_C)
#undef SV_C
    } else if (op.kind == SV_RZ || op.kind == SV_OP_PHASE) {
        const bool reg = op.kind == SV_RZ && ((rmask >> t0) & 1u);
        const bool one = op.kind == SV_OP_PHASE ? op.t[0] != 0 : ((base >> t0) & 1u) != 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const R im = ra_imdot<R>(l[v], p[v]);
            g += (reg ? ((v >> b0) & 1) : one) ? -im : im;
        }
    }
    ra_apply_op<R, RB>(p, op, rmask, base, cs, mats, true);
    ra_apply_op<R, RB>(l, op, rmask, base, cs, mats, true);
    return g;
}

// Hint: bring [p, p + bytes) into L2 (bytes a multiple of 16, p 16-byte aligned).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One amplitude (8 or 16 bytes) copied global -> shared asynchronously.
template <typename R>
__device__ __forceinline__ void cp_async_amp(void *dst, const Cx<R> *src) {
    if (sizeof(Cx<R>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Issue the copies of one gate-pass tile (swizzled layout) into shared memory.
template <typename R, typename E>
__device__ __forceinline__ void load_tile_async(E *tile, const Cx<R> *psi, uint64_t gbase,
                                                const uint64_t *hioff, int nlow, uint32_t T) {
    const uint32_t lowmask = (1u << nlow) - 1u;
    for (uint32_t j = threadIdx.x; j < T; j += blockDim.x)
        cp_async_amp<R>(&tile[swz_tile(j)], &psi[gbase | hioff[j >> nlow] | (j & lowmask)]);
}

// Shared-memory layout of a register-blocked pass (both kernels): the tiles,
// then these tables (offsets in bytes from the end of the tiles).
struct RegLayout {
    uint32_t hioff, cs, steps, blocks, mem, pbase, prb, acc, tot, sc, area, total;
};
// FP64 is 1/64 of the FP32 rate on this part: per-tile gradient partials stay
// in FP32 slots and reach FP64 once every kAdjFlush tiles
constexpr uint64_t kAdjFlush = 16;
__host__ __device__ inline uint32_t align16u(uint32_t v) { return (v + 15u) & ~15u; }
__host__ __device__ inline RegLayout reg_layout(const GatePassArgs &a, int amp, bool adj) {
    RegLayout L;
    const uint32_t nops = (uint32_t)(a.op_end - a.op_begin), nst = (uint32_t)(a.st_end - a.st_begin);
    const uint32_t nph = (uint32_t)(a.ph_end - a.ph_begin), nb = (uint32_t)(a.db_end - a.db_begin);
    uint32_t o = 0;
    L.hioff = o; o = align16u(o + 8u * (1u << (a.k - a.nlow)));
    L.cs = o;    o = align16u(o + (uint32_t)amp * nops);
    L.steps = o; o = align16u(o + 16u * nst);
    L.blocks = o; o = align16u(o + (uint32_t)sizeof(DiagBlock) * nb);
    L.mem = o;   o = align16u(o + (uint32_t)sizeof(DiagMember) * (uint32_t)(a.mem_end - a.mem_begin));
    L.pbase = o; o = align16u(o + 2u * kRegThreads * nph);
    L.prb = o;   o = align16u(o + 8u * nph);
    // adjoint gradient slots: per op and warp a partial of the state's real
    // type, and for complex64 an FP64 total per op (flushed every kAdjFlush tiles)
    L.acc = o;   o = align16u(o + (adj ? ((uint32_t)amp / 2u) * kAdjSlotStride * nops : 0u));
    L.tot = o;   o = align16u(o + (adj && amp == 8 ? 8u * nops : 0u));
    // factored RYs: per step the product of the factors applied before it
    // (adjoint), and the pass's total factor (entry nst)
    L.sc = o;    o = align16u(o + ((uint32_t)amp / 2u) * (nst + 1u));
    L.area = o;  o = align16u(o + (uint32_t)a.area);
    L.total = o;
    return L;
}

// Per-launch set-up shared by both kernels: high offsets, (cos, sin) per op
// (sin negated for the adjoint), steps, blocks, each phase's thread base and
// swizzled register-bit offsets, and the diagonal blocks' data (of D, or of
// D^dagger for the adjoint): a register block's table T[v][zm] and every
// thread's zm, a thread block's factor per thread.
template <typename R, int RB>
__device__ void reg_setup(unsigned char *sm, const RegLayout &L, const GatePassArgs &a, const DevOp *ops,
                          const Phase *phases, const RegStep *steps, const R *coef, const DiagBlock *dblocks,
                          const DiagMember *dmem, bool adj) {
    constexpr int V = 1 << RB;
    const int NT = blockDim.x, tid = threadIdx.x;
    uint64_t *hioff = reinterpret_cast<uint64_t *>(sm + L.hioff);
    Cx<R> *cs = reinterpret_cast<Cx<R> *>(sm + L.cs);
    RegStep *st = reinterpret_cast<RegStep *>(sm + L.steps);
    DiagBlock *bl = reinterpret_cast<DiagBlock *>(sm + L.blocks);
    uint16_t *pbase = reinterpret_cast<uint16_t *>(sm + L.pbase);
    uint16_t *prb = reinterpret_cast<uint16_t *>(sm + L.prb);
    const uint32_t nh = 1u << (a.k - a.nlow);
    for (uint32_t j = tid; j < nh; j += NT) hioff[j] = deposit(j, a.hi, a.nhi);
    for (int o = a.op_begin + tid; o < a.op_end; o += NT) {
        const int gi = ops[o].gate;
        cs[o - a.op_begin] = mk<R>(coef[2 * gi], adj ? -coef[2 * gi + 1] : coef[2 * gi + 1]);
    }
    __syncthreads();
    // the RYs of ROT steps as (t, factor), each step carrying their forms
    // (bit 8 + register bit set: form B)
    for (int s = a.st_begin + tid; s < a.st_end; s += NT) {
        RegStep S = steps[s];
        if (S.type == SV_STEP_ROT) {
            int o = S.op_begin;
            for (int b = 0; b < RB; ++b) {
                if (!((S.a >> b) & 1)) continue;
                const Cx<R> k = cs[o - a.op_begin];
                int fb;
                cs[o - a.op_begin] = ry_factored<R>(k.x, k.y, fb);
                if (fb) S.a |= 1 << (8 + b);
                ++o;
            }
        }
        st[s - a.st_begin] = S;
    }
    // prefix products of the factors in execution order (forward: ascending
    // steps; adjoint: descending), entry nst = the pass's total factor
    if (tid == 0) {
        R *sc = reinterpret_cast<R *>(sm + L.sc);
        const int nst = a.st_end - a.st_begin;
        R f = 1;
        for (int i = 0; i < nst; ++i) {
            const int s = adj ? a.st_end - 1 - i : a.st_begin + i;
            sc[s - a.st_begin] = f;
            const RegStep S = steps[s];
            if (S.type != SV_STEP_ROT) continue;
            for (int o = S.op_begin; o < S.op_end; ++o) {
                const int gi = ops[o].gate;
                const R c = coef[2 * gi], sn = adj ? -coef[2 * gi + 1] : coef[2 * gi + 1];
                int fb;
                f *= ry_factored<R>(c, sn, fb).y;
            }
        }
        sc[nst] = f;
    }
    for (int b = a.db_begin + tid; b < a.db_end; b += NT) bl[b - a.db_begin] = dblocks[b];
    DiagMember *mem = reinterpret_cast<DiagMember *>(sm + L.mem);
    for (int m = a.mem_begin + tid; m < a.mem_end; m += NT) mem[m - a.mem_begin] = dmem[m];
    for (int ph = a.ph_begin; ph < a.ph_end; ++ph) {
        const uint32_t rmask = phases[ph].rmask;
        const uint32_t base = phase_base(rmask, phases[ph].lanes, a.k);
        pbase[(ph - a.ph_begin) * NT + tid] = (uint16_t)base;
        if (tid < 4) {
            uint32_t rm = rmask, bitv = 0;
            for (int i = 0; i <= tid && rm; ++i) {
                bitv = rm & (0u - rm);
                rm ^= bitv;
            }
            prb[(ph - a.ph_begin) * 4 + tid] = (uint16_t)(tid < RB ? swz_tile(bitv) : 0u);
        }
    }
    unsigned char *area = sm + L.area;
    for (int b = a.db_begin; b < a.db_end; ++b) {
        const DiagBlock B = dblocks[b];
        const uint32_t base = phase_base(B.rmask, B.lanes, a.k);
        if (B.kind == 0) {
            Cx<R> *tab = reinterpret_cast<Cx<R> *>(area + B.smem);
            uint8_t *zmv = area + B.smem + V * V * (int)sizeof(Cx<R>);
            if (tid < V * V) {
                const int v = tid / V, zm = tid % V;
                Cx<R> r = mk<R>(((__popc((uint32_t)(v & zm)) & 1) ? -1 : 1), 0);
                for (int mi = B.m_begin; mi < B.m_end; ++mi) {
                    const DiagMember m = dmem[mi];
                    if (m.type == SV_DM_REG_RZ) {
                        const int gi = ops[m.op].gate;
                        const R c = coef[2 * gi], s = adj ? -coef[2 * gi + 1] : coef[2 * gi + 1];
                        r = cmul<R>(r, mk<R>(c, ((v >> m.a) & 1) ? s : -s));
                    } else if (m.type == SV_DM_REG_CZ) {
                        if ((v >> m.a) & (v >> m.b) & 1) r = mk<R>(-r.x, -r.y);
                    }
                }
                tab[v * V + zm] = r;
            }
            uint32_t zm = 0;
            for (int mi = B.m_begin; mi < B.m_end; ++mi) {
                const DiagMember m = dmem[mi];
                if (m.type == SV_DM_MIX_CZ && ((base >> m.b) & 1u)) zm ^= 1u << m.a;
            }
            zmv[tid] = (uint8_t)zm;
        } else {
            Cx<R> w = mk<R>(1, 0);
            for (int mi = B.m_begin; mi < B.m_end; ++mi) {
                const DiagMember m = dmem[mi];
                if (m.type == SV_DM_THR_RZ) {
                    const int gi = ops[m.op].gate;
                    const R c = coef[2 * gi], s = adj ? -coef[2 * gi + 1] : coef[2 * gi + 1];
                    w = cmul<R>(w, mk<R>(c, ((base >> m.a) & 1u) ? s : -s));
                } else if (m.type == SV_DM_THR_CZ) {
                    if ((base >> m.a) & (base >> m.b) & 1u) w = mk<R>(-w.x, -w.y);
                }
            }
            reinterpret_cast<Cx<R> *>(area + B.smem)[tid] = w;
        }
    }
}

// x[v] *= the block's factor (register block: table entry [v][zm]; thread block: one factor)
template <typename R, int RB>
__device__ __forceinline__ void reg_diag(RA<R> *x, const DiagBlock &B, const unsigned char *area) {
    constexpr int V = 1 << RB;
    if (B.kind == 0) {
        const Cx<R> *tab = reinterpret_cast<const Cx<R> *>(area + B.smem);
        const uint32_t zm = area[B.smem + V * V * (int)sizeof(Cx<R>) + threadIdx.x];
        const Cx<R> *col = tab + zm;
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = ra_cmul<R>(x[v], col[v * V]);
    } else {
        const Cx<R> w = reinterpret_cast<const Cx<R> *>(area + B.smem)[threadIdx.x];
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = ra_cmul<R>(x[v], w);
    }
}

// The same diagonal on two register sets (the adjoint's psi and lambda),
// each table entry loaded once.
template <typename R, int RB>
__device__ __forceinline__ void reg_diag2(RA<R> *x, RA<R> *y, const DiagBlock &B, const unsigned char *area) {
    constexpr int V = 1 << RB;
    if (B.kind == 0) {
        const Cx<R> *tab = reinterpret_cast<const Cx<R> *>(area + B.smem);
        const uint32_t zm = area[B.smem + V * V * (int)sizeof(Cx<R>) + threadIdx.x];
        const Cx<R> *col = tab + zm;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const Cx<R> w = col[v * V];
            x[v] = ra_cmul<R>(x[v], w);
            y[v] = ra_cmul<R>(y[v], w);
        }
    } else {
        const Cx<R> w = reinterpret_cast<const Cx<R> *>(area + B.smem)[threadIdx.x];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            x[v] = ra_cmul<R>(x[v], w);
            y[v] = ra_cmul<R>(y[v], w);
        }
    }
}

// The thread's 2^RB shared-memory indices of a phase (swizzled; the swizzle
// is linear, so index(base | sp[v]) = swz(base) ^ XOR of swz(register bits)).
template <int RB>
__device__ __forceinline__ void phase_slots(uint32_t *idx, uint32_t base, const uint16_t *prb) {
    idx[0] = swz_tile(base);
#pragma unroll
    for (int v = 1; v < (1 << RB); ++v) idx[v] = idx[v & (v - 1)] ^ prb[__ffs(v) - 1];
}

template <typename R, int RB>
__global__ void __launch_bounds__(512, 1) k_gate_reg(Cx<R> *__restrict__ psi, const GatePassArgs a,
                                                     const DevOp *__restrict__ ops, const Phase *__restrict__ phases,
                                                     const RegStep *__restrict__ steps, const R *__restrict__ coef,
                                                     const Cx<R> *__restrict__ mats,
                                                     const DiagBlock *__restrict__ dblocks,
                                                     const DiagMember *__restrict__ dmem) {
    constexpr int V = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t T = 1u << a.k;
    RA<R> *tiles = reinterpret_cast<RA<R> *>(smem);          // two tiles: the next one streams in
    unsigned char *sm = smem + 2 * T * sizeof(RA<R>);
    const RegLayout L = reg_layout(a, (int)sizeof(Cx<R>), false);
    reg_setup<R, RB>(sm, L, a, ops, phases, steps, coef, dblocks, dmem, false);
    __syncthreads();
    const R ftot = reinterpret_cast<const R *>(sm + L.sc)[a.st_end - a.st_begin];   // product of the RY factors
    const uint64_t *hioff = reinterpret_cast<const uint64_t *>(sm + L.hioff);
    const Cx<R> *cs = reinterpret_cast<const Cx<R> *>(sm + L.cs);
    const RegStep *st = reinterpret_cast<const RegStep *>(sm + L.steps);
    const DiagBlock *bl = reinterpret_cast<const DiagBlock *>(sm + L.blocks);
    const uint16_t *pbase = reinterpret_cast<const uint16_t *>(sm + L.pbase);
    const uint16_t *prb = reinterpret_cast<const uint16_t *>(sm + L.prb);
    const unsigned char *area = sm + L.area;
    const int NT = blockDim.x;
    const uint64_t ntiles = 1ull << a.nout;
    const uint32_t lowmask = (1u << a.nlow) - 1u;
    const uint64_t mine = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // tile bases walked with masked additions (current, and two ahead)
    const BitWalk bw = bit_walk(a.out, a.nout, gridDim.x);
    uint64_t base_pf = deposit(blockIdx.x, a.out, a.nout), base_cur = base_pf;
    for (uint64_t k = 0; k < 2; ++k) {
        if (k < mine) load_tile_async<R>(tiles + k * T, psi, base_pf, hioff, a.nlow, T);
        cp_async_commit();
        base_pf = walk_next(base_pf, bw);
    }
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t gbase = base_cur;
        base_cur = walk_next(base_cur, bw);
        RA<R> *tile = tiles + (it & 1) * T;
        cp_async_wait1();
        __syncthreads();
        for (int ph = a.ph_begin; ph < a.ph_end; ++ph) {
            const Phase P = phases[ph];
            const uint32_t base = pbase[(ph - a.ph_begin) * NT + threadIdx.x];
            uint32_t idx[V];
            phase_slots<RB>(idx, base, prb + (ph - a.ph_begin) * 4);
            RA<R> x[V];
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = tile[idx[v]];
            for (int s = P.st_begin; s < P.st_end; ++s) {
                const RegStep S = st[s - a.st_begin];
                if (S.type == SV_STEP_ROT) {
                    // factored RYs (t, factor): the factors are applied at the store
                    const Cx<R> *c = cs + (S.op_begin - a.op_begin);
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        if (!((S.a >> b) & 1)) continue;
                        const Cx<R> k = *c++;
                        ra_rotf_bit<R, V, RB>(x, b, (S.a >> (8 + b)) & 1, rotf<R>(k.x));
                    }
                } else if (S.type == SV_STEP_DIAG) {
                    reg_diag<R, RB>(x, bl[S.a - a.db_begin], area);
                } else {
                    DevOp op = ops[S.a];
                    if (has_out_target(op)) op = resolve_out(op, gbase);
                    ra_apply_op<R, RB>(x, op, P.rmask, base, cs[S.a - a.op_begin], mats, false);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) tile[idx[v]] = x[v];
            __syncthreads();
        }
        const Cx<R> *tc = reinterpret_cast<const Cx<R> *>(tile);
        for (uint32_t j = threadIdx.x; j < T; j += NT) {
            const Cx<R> v = tc[swz_tile(j)];
            psi[gbase | hioff[j >> a.nlow] | (j & lowmask)] = mk<R>(v.x * ftot, v.y * ftot);
        }
        __syncthreads();
        if (it + 2 < mine) load_tile_async<R>(tile, psi, base_pf, hioff, a.nlow, T);
        cp_async_commit();
        base_pf = walk_next(base_pf, bw);
    }
}

template <typename R, int RB>
__global__ void __launch_bounds__(512, 1) k_adj_reg(Cx<R> *__restrict__ psi, Cx<R> *__restrict__ lam,
                                                    const GatePassArgs a, const DevOp *__restrict__ ops,
                                                    const Phase *__restrict__ phases, const RegStep *__restrict__ steps,
                                                    const R *__restrict__ coef, const Cx<R> *__restrict__ mats,
                                                    double *__restrict__ part, int part_stride,
                                                    const DiagBlock *__restrict__ dblocks,
                                                    const DiagMember *__restrict__ dmem) {
    constexpr int V = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t T = 1u << a.k;
    const int nops = a.op_end - a.op_begin;
    const int NT = blockDim.x, nwarps = NT >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // slot row stride nwarps + 1: the lanes 0, 8, 16, 24 that add the four
    // gradients of a step (ops o .. o+3) hit four different banks
    const int AS = kAdjSlotStride;
    RA<R> *tl = reinterpret_cast<RA<R> *>(smem);           // lambda tile, then the psi tile
    RA<R> *tp = tl + T;
    unsigned char *sm = smem + 2 * T * sizeof(RA<R>);
    const RegLayout L = reg_layout(a, (int)sizeof(Cx<R>), true);
    R *acc = reinterpret_cast<R *>(sm + L.acc);
    double *tot64 = reinterpret_cast<double *>(sm + L.tot);
    for (int j = threadIdx.x; j < nops * AS; j += NT) acc[j] = 0;
    if constexpr (sizeof(R) == 4)
        for (int j = threadIdx.x; j < nops; j += NT) tot64[j] = 0.0;
    reg_setup<R, RB>(sm, L, a, ops, phases, steps, coef, dblocks, dmem, true);
    __syncthreads();
    // factored RYs: before step s both registers sets hold the true vectors
    // divided by scf[s], so a gradient part computed there is scaled by
    // scf[s]^2; the stores multiply by the total factor
    const R *scf = reinterpret_cast<const R *>(sm + L.sc);
    const R ftot = scf[a.st_end - a.st_begin];
    const uint64_t *hioff = reinterpret_cast<const uint64_t *>(sm + L.hioff);
    const Cx<R> *cs = reinterpret_cast<const Cx<R> *>(sm + L.cs);
    const RegStep *st = reinterpret_cast<const RegStep *>(sm + L.steps);
    const DiagBlock *bl = reinterpret_cast<const DiagBlock *>(sm + L.blocks);
    const uint16_t *pbase = reinterpret_cast<const uint16_t *>(sm + L.pbase);
    const uint16_t *prb = reinterpret_cast<const uint16_t *>(sm + L.prb);
    const unsigned char *area = sm + L.area;
    const DiagMember *mem = reinterpret_cast<const DiagMember *>(sm + L.mem);
    const uint64_t ntiles = 1ull << a.nout;
    const uint32_t lowmask = (1u << a.nlow) - 1u;
    const uint64_t mine = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const BitWalk bw = bit_walk(a.out, a.nout, gridDim.x);
    uint64_t gnext = deposit(blockIdx.x, a.out, a.nout);
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t gbase = gnext;
        gnext = walk_next(gnext, bw);
        if (it + 1 < mine) {
            // the next tile's psi and lambda runs head for L2 while this one is processed
            const uint64_t gn = gnext;
            const uint32_t runbytes = (1u << a.nlow) * (uint32_t)sizeof(Cx<R>);
            for (uint32_t j = threadIdx.x; j < (1u << (a.k - a.nlow)); j += NT) {
                prefetch_l2(psi + (gn | hioff[j]), runbytes);
                prefetch_l2(lam + (gn | hioff[j]), runbytes);
            }
        }
        {
            Cx<R> *tpc = reinterpret_cast<Cx<R> *>(tp), *tlc = reinterpret_cast<Cx<R> *>(tl);
            if (T == (uint32_t)(V * NT)) {
                // every load of the thread in flight before the first store
                Cx<R> vp[V], vl[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t j = threadIdx.x + (uint32_t)v * NT;
                    const uint64_t gi = gbase | hioff[j >> a.nlow] | (j & lowmask);
                    vp[v] = psi[gi];
                    vl[v] = lam[gi];
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t j = threadIdx.x + (uint32_t)v * NT;
                    tpc[swz_tile(j)] = vp[v];
                    tlc[swz_tile(j)] = vl[v];
                }
            } else {
                for (uint32_t j = threadIdx.x; j < T; j += NT) {
                    const uint64_t gi = gbase | hioff[j >> a.nlow] | (j & lowmask);
                    tpc[swz_tile(j)] = psi[gi];
                    tlc[swz_tile(j)] = lam[gi];
                }
            }
        }
        __syncthreads();
        for (int ph = a.ph_end - 1; ph >= a.ph_begin; --ph) {
            const Phase P = phases[ph];
            const uint32_t base = pbase[(ph - a.ph_begin) * NT + threadIdx.x];
            uint32_t idx[V];
            phase_slots<RB>(idx, base, prb + (ph - a.ph_begin) * 4);
            RA<R> xp[V], xl[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                xp[v] = tp[idx[v]];
                xl[v] = tl[idx[v]];
            }
            for (int s = P.st_end - 1; s >= P.st_begin; --s) {
                const RegStep S = st[s - a.st_begin];
                const R fs = scf[s - a.st_begin], fs2 = fs * fs;
                if (S.type == SV_STEP_ROT) {
                    // every RY of the step: gradient part at the step's end (they commute), then RY^dagger
                    R g[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        if (!((S.a >> b) & 1)) continue;
                        switch (b) {
                        case 0: g[0] = ra_ry_grad<R, V, 0>(xp, xl); break;
                        case 1: if constexpr (RB > 1) g[1] = ra_ry_grad<R, V, 1>(xp, xl); break;
                        case 2: if constexpr (RB > 2) g[2] = ra_ry_grad<R, V, 2>(xp, xl); break;
                        case 3: if constexpr (RB > 3) g[3] = ra_ry_grad<R, V, 3>(xp, xl); break;
                        default: break;
                        }
                    }
                    const R tot = warp_sum4<R>(g[0], g[1], g[2], g[3]) * fs2;
                    const Cx<R> *c = cs + (S.op_begin - a.op_begin);
                    int o = S.op_begin - a.op_begin;
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        if (!((S.a >> b) & 1)) continue;
                        if (lane == 8 * b) acc[o * AS + warp] += tot;
                        ++o;
                        const Cx<R> k = *c++;
                        const RotF<R> rk = rotf<R>(k.x);
                        const bool fb = (S.a >> (8 + b)) & 1;
                        ra_rotf_bit<R, V, RB>(xp, b, fb, rk);
                        ra_rotf_bit<R, V, RB>(xl, b, fb, rk);
                    }
                } else if (S.type == SV_STEP_DIAG) {
                    // every RZ member's generator expectation at the block's end (Z
                    // commutes with the block), then D^dagger on both register sets
                    const DiagBlock B = bl[S.a - a.db_begin];
                    R tv[V], tot = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        tv[v] = ra_imdot<R>(xl[v], xp[v]);
                        tot += tv[v];
                    }
                    if (B.kind == 0) {
                        R sb[4] = {0, 0, 0, 0};
                        signed_bit_sums<R, RB>(tv, sb);
                        const R red = warp_sum4<R>(sb[0], sb[1], sb[2], sb[3]) * fs2;
                        for (int mi = B.m_begin; mi < B.m_end; ++mi) {
                            const DiagMember m = mem[mi - a.mem_begin];
                            if (m.type == SV_DM_REG_RZ && lane == 8 * m.a)
                                acc[(m.op - a.op_begin) * AS + warp] += red;
                        }
                    } else {
                        // thread RZ members: +-tot by the thread's bit, four at a time
                        for (int m0 = B.m_begin; m0 < B.m_end; m0 += 4) {
                            R vals[4] = {0, 0, 0, 0};
                            int opi[4] = {-1, -1, -1, -1};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (m0 + j < B.m_end) {
                                    const DiagMember m = mem[m0 + j - a.mem_begin];
                                    if (m.type == SV_DM_THR_RZ) {
                                        vals[j] = ((base >> m.a) & 1u) ? -tot : tot;
                                        opi[j] = m.op - a.op_begin;
                                    }
                                }
                            }
                            const R red = warp_sum4<R>(vals[0], vals[1], vals[2], vals[3]) * fs2;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (lane == 8 * j && opi[j] >= 0) acc[opi[j] * AS + warp] += red;
                        }
                    }
                    reg_diag2<R, RB>(xp, xl, B, area);
                } else {
                    DevOp op = ops[S.a];
                    if (has_out_target(op)) op = resolve_out(op, gbase);
                    R g = ra_adjoint_op<R, RB>(xp, xl, op, P.rmask, base, cs[S.a - a.op_begin], mats);
                    if (has_param(op.kind)) {
                        g = warp_sum<R>(g) * fs2;
                        if (lane == 0) acc[(S.a - a.op_begin) * AS + warp] += g;
                    }
                }
            }
            // the slots again (fewer registers live across the steps)
            phase_slots<RB>(idx, pbase[(ph - a.ph_begin) * NT + threadIdx.x], prb + (ph - a.ph_begin) * 4);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                tp[idx[v]] = xp[v];
                tl[idx[v]] = xl[v];
            }
            __syncthreads();
        }
        {
            const Cx<R> *tpc = reinterpret_cast<const Cx<R> *>(tp), *tlc = reinterpret_cast<const Cx<R> *>(tl);
            for (uint32_t j = threadIdx.x; j < T; j += NT) {
                const uint64_t gi = gbase | hioff[j >> a.nlow] | (j & lowmask);
                const Cx<R> p = tpc[swz_tile(j)], l = tlc[swz_tile(j)];
                psi[gi] = mk<R>(p.x * ftot, p.y * ftot);
                lam[gi] = mk<R>(l.x * ftot, l.y * ftot);
            }
        }
        __syncthreads();
        if constexpr (sizeof(R) == 4) {
            // the next writes to the slots follow the next tile's barrier
            if (((it + 1) % kAdjFlush) == 0 || it + 1 == mine) {
                for (int o = threadIdx.x; o < nops; o += NT) {
                    float f = 0.f;
                    for (int w = 0; w < nwarps; ++w) {
                        f += acc[o * AS + w];
                        acc[o * AS + w] = 0.f;
                    }
                    tot64[o] += (double)f;
                }
            }
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nops; o += NT) {
        double tsum = 0.0;
        if constexpr (sizeof(R) == 4) tsum = tot64[o];
        else
            for (int w = 0; w < nwarps; ++w) tsum += acc[o * AS + w];
        part[(size_t)blockIdx.x * part_stride + a.op_begin + o] = tsum;
    }
}
#undef SV_RB_SWITCH

// -------------------------------------------------------------------- K-QR --
struct SwapArgs {
    int n, L, ntb, nlo, nhi, nout;
    int8_t tb[24];           // physical bits of tile bits L..ntb-1
    int8_t la[40], lb[40];   // tile-bit pairs swapped inside a tile
    int8_t ha[40], hb[40];   // physical pairs outside the tile (tile <-> partner tile)
    int8_t out[64];          // physical bits outside the tile, ascending
};

__device__ __forceinline__ uint32_t sigma_lo(uint32_t j, const SwapArgs &a) {
    for (int i = 0; i < a.nlo; ++i)
        if (((j >> a.la[i]) ^ (j >> a.lb[i])) & 1u) j ^= (1u << a.la[i]) | (1u << a.lb[i]);
    return j;
}
__device__ __forceinline__ uint64_t sigma_hi(uint64_t b, const SwapArgs &a) {
    for (int i = 0; i < a.nhi; ++i)
        if (((b >> a.ha[i]) ^ (b >> a.hb[i])) & 1ull) b ^= (1ull << a.ha[i]) | (1ull << a.hb[i]);
    return b;
}

// Element x moves to x with every paired bit exchanged.  A CTA takes a tile
// -- the lowest L index bits (one contiguous run) plus the partners of paired
// run bits -- and, when pairs lie outside the tile, its partner tile; both
// are loaded before either is written, so the swap is in place.  Tiles whose
// pairs agree everywhere are not touched.  Global accesses are 16-byte vectors
// along the run; shared memory is swizzled so that the bit exchanges of a
// warp's reads spread over the banks.
template <typename R>
__device__ __forceinline__ uint32_t swz(uint32_t j) {
    // XOR bits 1..3 (c64) or 0..2 (c128) of the index with higher bits: a
    // bijection that keeps 16-byte pairs of complex64 adjacent
    if (sizeof(R) == 4) return j ^ ((((j >> 4) ^ (j >> 8)) & 7u) << 1);
    return j ^ (((j >> 3) ^ (j >> 6)) & 7u);
}

template <typename R>
__global__ void __launch_bounds__(256) k_bitswap(Cx<R> *__restrict__ psi, const SwapArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int VEC = 16 / sizeof(Cx<R>);        // amplitudes per 16-byte access
    const uint32_t T = 1u << a.ntb;
    const uint32_t nh = 1u << (a.ntb - a.L);
    Cx<R> *A = reinterpret_cast<Cx<R> *>(smem);
    Cx<R> *B = A + T;
    uint64_t *hioff = reinterpret_cast<uint64_t *>(B + T);
    // source slot (swizzled, after the in-tile exchanges) of every tile index,
    // two 16-bit entries per 32-bit word: computed once per CTA
    uint32_t *pt = reinterpret_cast<uint32_t *>(hioff + nh);
    for (uint32_t j = threadIdx.x; j < nh; j += blockDim.x) hioff[j] = deposit(j, a.tb, a.ntb - a.L);
    for (uint32_t q = threadIdx.x; q < T / 2; q += blockDim.x)
        pt[q] = swz<R>(sigma_lo(2 * q, a)) | (swz<R>(sigma_lo(2 * q + 1, a)) << 16);
    __syncthreads();
    const uint32_t runmask = (1u << a.L) - 1u;
    const uint64_t ntiles = 1ull << a.nout;
    const bool vec = (VEC == 2) && a.L >= 1;
    // no in-tile exchange moves bit 0: the source slots of a 16-byte pair are
    // adjacent (the swizzle keeps bit 0), so the pair is one 16-byte load
    bool bit0_fixed = true;
    for (int i = 0; i < a.nlo; ++i)
        if (a.la[i] == 0 || a.lb[i] == 0) bit0_fixed = false;
    const BitWalk bw = bit_walk(a.out, a.nout, gridDim.x);
    uint64_t bnext = deposit(blockIdx.x, a.out, a.nout);
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const uint64_t b0 = bnext;
        bnext = walk_next(bnext, bw);
        const uint64_t b1 = sigma_hi(b0, a);
        if (b1 < b0) continue;
        const bool self = (b1 == b0);
        if (self && a.nlo == 0) continue;
        if (vec) {
            // 16-byte copies straight into shared memory (j even and bit 0 of b0, b1 clear: both ends aligned)
            for (uint32_t j = 2 * threadIdx.x; j < T; j += 2 * blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s = swz<R>(j);
                cp_async16(&A[s], &psi[b0 | off]);
                if (!self) cp_async16(&B[s], &psi[b1 | off]);
            }
            cp_async_commit();
            cp_async_wait0();
        } else {
            for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s = swz<R>(j);
                A[s] = psi[b0 | off];
                if (!self) B[s] = psi[b1 | off];
            }
        }
        __syncthreads();
        if (vec && bit0_fixed) {
            for (uint32_t j = 2 * threadIdx.x; j < T; j += 2 * blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s0 = pt[j >> 1] & 0xFFFFu;
                const Cx<R> *src = self ? A : B;
                *reinterpret_cast<float4 *>(&psi[b0 | off]) = *reinterpret_cast<const float4 *>(&src[s0]);
                if (!self)
                    *reinterpret_cast<float4 *>(&psi[b1 | off]) = *reinterpret_cast<const float4 *>(&A[s0]);
            }
        } else if (vec) {
            for (uint32_t j = 2 * threadIdx.x; j < T; j += 2 * blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t pp = pt[j >> 1], s0 = pp & 0xFFFFu, s1 = pp >> 16;
                const Cx<R> *src = self ? A : B;
                float4 v;
                v.x = src[s0].x; v.y = src[s0].y; v.z = src[s1].x; v.w = src[s1].y;
                *reinterpret_cast<float4 *>(&psi[b0 | off]) = v;
                if (!self) {
                    float4 u;
                    u.x = A[s0].x; u.y = A[s0].y; u.z = A[s1].x; u.w = A[s1].y;
                    *reinterpret_cast<float4 *>(&psi[b1 | off]) = u;
                }
            }
        } else {
            for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s = (j & 1) ? (pt[j >> 1] >> 16) : (pt[j >> 1] & 0xFFFFu);
                psi[b0 | off] = self ? A[s] : B[s];
                if (!self) psi[b1 | off] = A[s];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- staged cosets --
// A coset is staged with 16-byte cp.async copies spread over all threads
// (runs are >= 16 bytes and contiguous); two buffers alternate so the next
// coset's copies are in flight while the current one is processed
// (commit/wait groups: at iteration i, groups i and i+1 are outstanding and
// waiting for all but the newest completes coset i).

template <typename R>
__device__ __forceinline__ void load_coset(Cx<R> *dst, const Cx<R> *psi, uint64_t rep, const uint64_t *spanv, int kl,
                                           uint32_t E) {
    constexpr uint32_t PER = 16 / sizeof(Cx<R>);
    const uint32_t lowmask = (1u << kl) - 1u;
    for (uint32_t q = threadIdx.x; q < E / PER; q += blockDim.x) {
        const uint32_t e = q * PER;
        cp_async16(dst + e, psi + (rep ^ spanv[e >> kl] ^ (e & lowmask)));
    }
}

__device__ __forceinline__ void coset_span(const CosetArgs &a, uint64_t *spanv) {
    const uint32_t M = 1u << a.m;
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        uint64_t v = 0;
        for (int i = 0; i < a.m; ++i)
            if (j >> i & 1u) v ^= a.basis[i];
        spanv[j] = v;
    }
    __syncthreads();
}

// ------------------------------------------------------------------- K-EVC --
// For group x (offset X inside the staged coset, X = (c << kl) | xlo) and
// each pair (b, b^x), w = conj(psi[b^x]) psi[b]; string (x, z) with
// nY = |x & z| contributes 2 Re(i^nY (-1)^{|b&z|} w) per pair.  The formula
// gives the same value from either element of the pair (swapping the roles
// conjugates w and flips the sign by (-1)^nY, which cancel), so each pair is
// evaluated once by whichever thread the split below assigns it to.  x = 0
// contributes (-1)^{|b&z|} |psi[b]|^2 per element.  b is the FULL physical
// index, so Z on chunk bits gives the per-chunk sign s_j of Eq. par_exp.
//
// Thread mapping: thread t owns the staged elements e = t + j*NT, j < EPT
// (held in registers), i.e. run position l = t mod 2^kl and run index
// a = a0 + j*astep with a0 = t >> kl, astep = NT >> kl.  Because parity is
// linear, parity(b & z) = parity((rep|l) & z) ^ parity(a0 & bz) ^
// parity(j & w), bz = parities of the span basis against z, w = bz >> log2(astep);
// the last term over all j is one 32-bit Walsh mask per string.
// Pair split: partner in the same thread (c's lowest bit among the j bits):
// take j with that bit clear; partner in another thread (c's lowest bit among
// the a0 bits, or x inside the run): the thread whose own bit is 0 takes the
// first half of its j, its partner the second half.
constexpr int kEvcChunk = 4;   // strings of one group evaluated together

__device__ __forceinline__ uint32_t walsh_mask(uint32_t w) {
    uint32_t m = 0;
    if (w & 1u) m ^= 0xAAAAAAAAu;
    if (w & 2u) m ^= 0xCCCCCCCCu;
    if (w & 4u) m ^= 0xF0F0F0F0u;
    if (w & 8u) m ^= 0xFF00FF00u;
    if (w & 16u) m ^= 0xFFFF0000u;
    return m;
}

struct ThreadCoset {
    uint32_t l, a0, ash;   // run position, first run index, log2(astep)
};

__device__ __forceinline__ ThreadCoset thread_coset(int kl) {
    ThreadCoset tc;
    tc.l = threadIdx.x & ((1u << kl) - 1u);
    tc.a0 = threadIdx.x >> kl;
    tc.ash = (uint32_t)(__ffs(blockDim.x) - 1) - (uint32_t)kl;
    return tc;
}

// j selection of the pair split (EPT = elements per thread): a mask of the
// thread's elements that takes exactly one element of every pair, half of
// them per thread; *fac = 2.  If no such split exists (c flips every j bit
// while its lowest bit is among the a0 bits) all elements are taken and
// *fac = 1 (every element then evaluates its own term).
__device__ __forceinline__ uint32_t pair_select(const ThreadCoset &tc, uint32_t X, int kl, int ept, int &fac) {
    const uint32_t all = ept >= 32 ? 0xFFFFFFFFu : ((1u << ept) - 1u);
    const int jb = __ffs(ept) - 1;                 // log2(ept)
    const uint32_t c = X >> kl;
    fac = 2;
    if (c) {
        const int cb = __ffs(c) - 1;
        if (cb >= (int)tc.ash) return all & ~walsh_mask(1u << (cb - tc.ash));   // partner: same thread
        const uint32_t cj = c >> tc.ash;                                         // j bits flipped by c
        for (int h = 0; h < jb; ++h)
            if (!((cj >> h) & 1u)) {
                const uint32_t ph = walsh_mask(1u << h);
                return all & (((tc.a0 >> cb) & 1u) ? ph : ~ph);
            }
        fac = 1;
        return all;
    }
    const int pl = __ffs(X) - 1;   // x inside the run: partner = l ^ xlo, same j
    if (jb == 0) { fac = 1; return all; }
    const uint32_t ph = walsh_mask(1u);
    return all & (((tc.l >> pl) & 1u) ? ph : ~ph);
}

// The same split as (h, s): take the elements j whose bit h equals s, or
// every element (h = -1, factor 1).
struct PairSel {
    int h, s, fac;
};

__device__ __forceinline__ PairSel pair_split(const ThreadCoset &tc, uint32_t X, int kl, int ept) {
    const int jb = __ffs(ept) - 1;
    const uint32_t c = X >> kl;
    if (c) {
        const int cb = __ffs(c) - 1;
        if (cb >= (int)tc.ash) return {cb - (int)tc.ash, 0, 2};
        const uint32_t cj = c >> tc.ash;
        for (int h = 0; h < jb; ++h)
            if (!((cj >> h) & 1u)) return {h, (int)((tc.a0 >> cb) & 1u), 2};
        return {-1, 0, 1};
    }
    if (jb == 0) return {-1, 0, 1};
    return {0, (int)((tc.l >> (__ffs(X) - 1)) & 1u), 2};
}

// val with its sign flipped when bit j of sm is set.
template <int J>
__device__ __forceinline__ float flip_bit(float v, uint32_t sm) {
    return __int_as_float(__float_as_int(v) ^ (int)((sm << (31 - J)) & 0x80000000u));
}
template <int J>
__device__ __forceinline__ double flip_bit(double v, uint32_t sm) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)((sm >> J) & 1u) << 63));
}

// +1 or -1 by bit i of w.
template <typename R>
__device__ __forceinline__ R sign_of_bit(uint32_t w, int i) {
    return ((w >> i) & 1u) ? (R)-1 : (R)1;
}

// sum_j (-1)^{parity(j & w)} val[j] over N = 2^L values, as the Walsh-Hadamard
// butterfly restricted to one output: level i folds pairs differing in bit i
// with one fused multiply-add by the sign of bit i of w (log2 N levels, N - 1
// operations, no per-element sign work).
template <typename R, int N>
__device__ __forceinline__ R walsh_sum(R *val, uint32_t w) {
#pragma unroll
    for (int i = 0, n = N; n > 1; ++i, n >>= 1) {
        const R sg = sign_of_bit<R>(w, i);
#pragma unroll
        for (int k = 0; k < n / 2; ++k) val[k] = fma(sg, val[2 * k + 1], val[2 * k]);
    }
    return val[0];
}

// Sum over the selected elements j = (j' with bit S inserted at H) of the
// pair term Re or Im(conj(partner) own), signed by (-1)^{parity(j & w)}.
// NT = 2^LOGNT, E = EPT*NT.
template <typename R, int EPT, int H, int S, bool ODD, int LOGNT>
__device__ __forceinline__ R evc_sel_loop(const Cx<R> *t, const Cx<R> *own, uint32_t X, uint32_t w) {
    constexpr int SH = LOGNT + (sizeof(R) == 4 ? 3 : 4);
    R val[EPT / 2];
    // partner of element j: byte offset B ^ (j << SH) of the staged coset
    const uint32_t sb = smem_u32(t);
    const uint32_t B = (threadIdx.x ^ X) * (uint32_t)sizeof(Cx<R>);
#pragma unroll
    for (int jp = 0; jp < EPT / 2; ++jp) {
        const int j = ((jp >> H) << (H + 1)) | (S << H) | (jp & ((1 << H) - 1));
        const Cx<R> u = own[j];
        const Cx<R> v = lds_cx<R>(sb + (B ^ ((uint32_t)j << SH)));
        val[jp] = ODD ? (v.x * u.y - v.y * u.x) : (v.x * u.x + v.y * u.y);
    }
    // parity(j & w) = (S & w_H) ^ parity(j' & w'), w' = w with bit H removed
    const uint32_t wp = (w & ((1u << H) - 1u)) | ((w >> (H + 1)) << H);
    const R r = walsh_sum<R, EPT / 2>(val, wp);
    return (S && ((w >> H) & 1u)) ? -r : r;
}

template <typename R, int EPT, bool ODD, int LOGNT>
__device__ __forceinline__ R evc_all_loop(const Cx<R> *t, const Cx<R> *own, uint32_t X, uint32_t w) {
    constexpr int SH = LOGNT + (sizeof(R) == 4 ? 3 : 4);
    R val[EPT];
    const uint32_t sb = smem_u32(t);
    const uint32_t B = (threadIdx.x ^ X) * (uint32_t)sizeof(Cx<R>);
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const Cx<R> u = own[j];
        if (X) {
            const Cx<R> v = lds_cx<R>(sb + (B ^ ((uint32_t)j << SH)));
            val[j] = ODD ? (v.x * u.y - v.y * u.x) : (v.x * u.x + v.y * u.y);
        } else {
            val[j] = u.x * u.x + u.y * u.y;
        }
    }
    return walsh_sum<R, EPT>(val, w);
}

// Fast path (NT = 2^LOGNT, E = EPT * NT): one switch on the pass code
// (h + 1) | s << 3 | odd << 4 of the pair split (h = -1: every element); the
// result is signed by (-1)^{parity(j & w)} per element j.
template <typename R, int EPT, int LOGNT>
__device__ __forceinline__ R evc_fast(const Cx<R> *t, const Cx<R> *own, uint32_t X, uint32_t code, uint32_t w) {
    switch (code) {
    case 0: return evc_all_loop<R, EPT, false, LOGNT>(t, own, X, w);
    case 16: return evc_all_loop<R, EPT, true, LOGNT>(t, own, X, w);
#define SV_SEL(HH, SS, OO)                                                                               \
    case (HH + 1) | (SS << 3) | (OO << 4):                                                               \
        if constexpr ((1 << (HH + 1)) <= EPT) return evc_sel_loop<R, EPT, HH, SS, OO != 0, LOGNT>(t, own, X, w); \
        else return (R)0;
#define SV_SEL4(HH) SV_SEL(HH, 0, 0) SV_SEL(HH, 1, 0) SV_SEL(HH, 0, 1) SV_SEL(HH, 1, 1)
    SV_SEL4(0) SV_SEL4(1) SV_SEL4(2) SV_SEL4(3)
#undef SV_SEL4
#undef SV_SEL
    default: return (R)0;
    }
}

// Large groups (complex64, 16 amplitudes per thread, 512 threads, 8192
// staged): instead of a signed sum per string, the coset's pair terms
// val(b) = Re or Im of conj(psi[b^x]) psi[b] (every b, each pair from both
// sides) are Walsh-Hadamard transformed over the element bits (in registers)
// and the lane bits (shuffles); the 16 warps' partial transforms go to
// shared memory, and the thread owning string s finishes its one
// coefficient with a 16-term signed sum over the warp bits.  Because
// parity(b & z) = parity(rep & z) ^ parity(t & tau) ^ parity(j & w) with
// tau = (z mod 2^kl) | (bz mod 2^ash) << kl, string s needs the coefficient
// at element frequency w, lane frequency tau mod 32 and warp frequency
// tau >> 5.  Cost per coset: one transform per group and needed part (Re,
// Im), independent of the group's string count.
// Walsh fold of N = 2^L values without touching them: sum_j (-1)^{parity(j & w)} val[j].
template <typename R, int N>
__device__ __forceinline__ R walsh_sum_ro(const R *val, uint32_t w) {
    R tmp[N / 2];
    const R s0 = sign_of_bit<R>(w, 0);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) tmp[k] = fma(s0, val[2 * k + 1], val[2 * k]);
#pragma unroll
    for (int i = 1, n = N / 2; n > 1; ++i, n >>= 1) {
        const R sg = sign_of_bit<R>(w, i);
#pragma unroll
        for (int k = 0; k < n / 2; ++k) tmp[k] = fma(sg, tmp[2 * k + 1], tmp[2 * k]);
    }
    return tmp[0];
}

// Per-string constants of a general EVC pass (complex64 transform-capable
// passes), staged once per CTA: the signs of the element Walsh fold per level
// (frequency w = bz >> log2(512 / 2^kl), with the pair-split bit removed when
// the group splits), z, the thread-sign mask tz (parity(tid & tz) =
// parity(l & z) ^ parity(a0 & bz)) and flags: bit 0 the part (nY odd: Im),
// bit 1 the i^nY sign, bit 2 the split bit of w.
struct StrC {
    float4 lev;
    uint64_t z;
    uint32_t tz, flags;
};
static_assert(sizeof(StrC) == 32, "StrC layout");

template <int N>
__device__ __forceinline__ float walsh_lev(const float *val, const float4 &lev) {
    const float sg[4] = {lev.x, lev.y, lev.z, lev.w};
    float tmp[N / 2];
#pragma unroll
    for (int k = 0; k < N / 2; ++k) tmp[k] = fmaf(sg[0], val[2 * k + 1], val[2 * k]);
#pragma unroll
    for (int i = 1, n = N / 2; n > 1; ++i, n >>= 1) {
#pragma unroll
        for (int k = 0; k < n / 2; ++k) tmp[k] = fmaf(sg[i], tmp[2 * k + 1], tmp[2 * k]);
    }
    return tmp[0];
}

// Re and Im of conj(partner) * own for the thread's 16 elements (complex64,
// 512 threads): partner of element j is t[(tid + 512 j) ^ X]; X = 0 gives
// |own|^2 and 0.
__device__ __forceinline__ void pair_terms_all(const float2 *t, const float2 *own, uint32_t X, float *vr, float *vi) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float2 u = own[j];
        if (X) {
            const float2 w = t[(threadIdx.x + j * 512u) ^ X];
            vr[j] = w.x * u.x + w.y * u.y;
            vi[j] = w.x * u.y - w.y * u.x;
        } else {
            vr[j] = u.x * u.x + u.y * u.y;
            vi[j] = 0.f;
        }
    }
}
// The same for the 8 elements j with bit H of j equal to S (one element of
// every pair), as j' = j with bit H removed.
template <int H, int S>
__device__ __forceinline__ void pair_terms_sel(const float2 *t, const float2 *own, uint32_t X, float *vr, float *vi) {
    const uint32_t sb = smem_u32(t);
    const uint32_t B = ((threadIdx.x ^ X) * 8u) ^ ((uint32_t)S << (H + 12));
#pragma unroll
    for (int jp = 0; jp < 8; ++jp) {
        const int j0 = ((jp >> H) << (H + 1)) | (jp & ((1 << H) - 1));
        const float2 u = own[j0 | (S << H)];
        const float2 w = lds_cx<float>(sb + (B ^ ((uint32_t)j0 << 12)));
        vr[jp] = w.x * u.x + w.y * u.y;
        vi[jp] = w.x * u.y - w.y * u.x;
    }
}

constexpr int kXformMinStrings = 16;  // groups with at least this many strings take the transform path
// shared-memory layout of k_evc_pass: two staged cosets, the span table, per
// string and warp a partial of the state's real type (FP64 is 1/64 of the
// FP32 rate here: complex64 partials reach an FP64 total per string every
// kEvcFlush cosets), then the transform scratch and string constants
constexpr uint64_t kEvcFlush = 64;
__host__ __device__ inline size_t evc_al16(size_t v) { return (v + 15) & ~(size_t)15; }
__host__ __device__ inline size_t evc_span_end(uint32_t E, int m, size_t rbytes) {
    return evc_al16(2 * (size_t)E * 2 * rbytes + ((size_t)8 << m));
}
__host__ __device__ inline size_t evc_part_bytes(int nslots, int nwarps, size_t rbytes) {
    return evc_al16((size_t)nslots * nwarps * rbytes);
}
__host__ __device__ inline size_t evc_slot_bytes(int nslots, int nwarps, size_t rbytes) {
    return evc_part_bytes(nslots, nwarps, rbytes) + (rbytes == 4 ? evc_al16((size_t)nslots * 8) : 0);
}
constexpr int kXformScratch = 8192;   // floats of shared scratch (16 element x 16 warp x 32 lane frequencies)

__device__ __forceinline__ void xform_part(float *v, float *scr, const float *lsg) {
    // element bits: in-register butterflies (natural-order output)
#pragma unroll
    for (int h = 1; h < 16; h <<= 1)
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (!(i & h)) {
                const float x = v[i], y = v[i + h];
                v[i] = x + y;
                v[i + h] = x - y;
            }
    // lane bits: the lower lane of a pair keeps x + y, the upper y - x... as fma(sign, own, partner)
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaf(lsg[b], v[i], __shfl_xor_sync(0xffffffffu, v[i], 1 << b));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 16; ++i) scr[(i * 16 + warp) * 32 + lane] = v[i];
}

// Owner side: coefficient (fj, fw, fl) of the scratch, finished over the warp bits.
__device__ __forceinline__ float xform_coef(const float *scr, uint32_t fj, uint32_t fw, uint32_t fl) {
    float c[16];
#pragma unroll
    for (int w = 0; w < 16; ++w) c[w] = scr[(fj * 16 + w) * 32 + fl];
    return walsh_sum<float, 16>(c, fw);
}

template <typename R, int EPT>
__global__ void __launch_bounds__(512, 1) k_evc_pass(const Cx<R> *__restrict__ psi, const CosetArgs a,
                                                     const DevGroup *__restrict__ groups,
                                                     const DevString *__restrict__ strs, double *__restrict__ part,
                                                     int part_stride, int xform) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    const int nslots = a.s_end - a.s_begin;
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Cx<R> *buf = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(buf + 2 * E);
    unsigned char *slots = smem + evc_span_end(E, a.m, sizeof(R));
    R *acc = reinterpret_cast<R *>(slots);                                 // [string][warp] partials
    double *tot64 = reinterpret_cast<double *>(slots + evc_part_bytes(nslots, nwarps, sizeof(R)));
    float *scr = reinterpret_cast<float *>(slots + evc_slot_bytes(nslots, nwarps, sizeof(R)));   // transform scratch (when xform)
    StrC *strc = reinterpret_cast<StrC *>(scr + kXformScratch);         // per-string constants (when xform)
    for (int j = threadIdx.x; j < nslots * nwarps; j += blockDim.x) acc[j] = 0;
    if constexpr (sizeof(R) == 4)
        for (int j = threadIdx.x; j < nslots; j += blockDim.x) tot64[j] = 0.0;
    coset_span(a, spanv);
    const ThreadCoset tc = thread_coset(a.kl);
    // the transform path needs complex64, 16 per thread, 512 threads, 8192 staged, the scratch
    bool use_x = false;
    float lsg[5] = {1.f, 1.f, 1.f, 1.f, 1.f};
    if constexpr (sizeof(R) == 4 && EPT == 16) {
        use_x = xform && blockDim.x == 512 && E == 8192u;
        for (int b = 0; b < 5; ++b) lsg[b] = ((lane >> b) & 1) ? -1.f : 1.f;
        if (use_x) {
            // the pair-split bit of a group is the same in every thread (only its side differs)
            for (int gi = a.g_begin + warp; gi < a.g_end; gi += nwarps) {
                const DevGroup G = groups[gi];
                const int h = G.X ? pair_split(tc, G.X, a.kl, 16).h : -1;
                for (int q = G.s_begin + lane; q < G.s_end; q += 32) {
                    const DevString S = strs[q];
                    const uint32_t w = S.bz >> tc.ash;
                    uint32_t wf = w, flip = 0;
                    if (h >= 0) {
                        wf = (w & ((1u << h) - 1u)) | ((w >> (h + 1)) << h);
                        flip = (w >> h) & 1u;
                    }
                    StrC c;
                    c.lev = make_float4((wf & 1u) ? -1.f : 1.f, (wf & 2u) ? -1.f : 1.f, (wf & 4u) ? -1.f : 1.f,
                                        (wf & 8u) ? -1.f : 1.f);
                    c.z = S.z;
                    c.tz = (uint32_t)(S.z & ((1ull << a.kl) - 1ull)) | ((S.bz & ((1u << tc.ash) - 1u)) << a.kl);
                    const uint32_t neg0 = G.X ? (uint32_t)((S.nY == 1) | (S.nY == 2)) : 0u;
                    c.flags = (uint32_t)(S.nY & 1) | (neg0 << 1) | (flip << 2);
                    strc[q - a.s_begin] = c;
                }
            }
        }
    }
    const uint64_t ncos = 1ull << a.nfree;
    const uint64_t mine = blockIdx.x < ncos ? (ncos - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // coset representatives walked with masked additions: rep_cur of the
    // current iteration, rep_pf of the one two ahead (the next copy issued)
    const BitWalk bw = bit_walk(a.freeb, a.nfree, gridDim.x);
    uint64_t rep_pf = deposit(blockIdx.x, a.freeb, a.nfree), rep_cur = rep_pf;
    for (uint64_t k = 0; k < 2; ++k) {
        if (k < mine) load_coset<R>(buf + k * E, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t rep = rep_cur;
        rep_cur = walk_next(rep_cur, bw);
        Cx<R> *t = buf + (it & 1) * E;
        cp_async_wait1();
        __syncthreads();
        Cx<R> own[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = threadIdx.x + j * blockDim.x;
            own[j] = e < E ? t[e] : mk<R>(0, 0);
        }
        for (int gi = a.g_begin; gi < a.g_end; ++gi) {
            const DevGroup G = groups[gi];
            if constexpr (sizeof(R) == 4 && EPT == 16) {
                const int K = G.s_end - G.s_begin;
                if (use_x && K < kXformMinStrings) {
                    // up to 15 strings: the Re and Im pair terms of the thread's elements once
                    // (one element of every pair when the split allows, else all of them),
                    // then per string a Walsh fold and the thread / coset sign; four
                    // strings share one warp reduction
                    const PairSel ps = G.X ? pair_split(tc, G.X, a.kl, 16) : PairSel{-1, 0, 1};
                    float vr[16], vi[16];
#define SV_PT(HH) \
    case HH: if (ps.s) pair_terms_sel<HH, 1>(t, own, G.X, vr, vi); else pair_terms_sel<HH, 0>(t, own, G.X, vr, vi); break;
                    switch (ps.h) {
                        SV_PT(0) SV_PT(1) SV_PT(2) SV_PT(3)
                    default: pair_terms_all(t, own, G.X, vr, vi); break;
                    }
#undef SV_PT
                    const float fac = (float)ps.fac;
                    const bool split = ps.h >= 0;
                    for (int q0 = G.s_begin; q0 < G.s_end; q0 += 4) {
                        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (q0 + k < G.s_end) {
                                const StrC C = strc[q0 + k - a.s_begin];
                                float r;
                                if (split) {
                                    // the fold over j' (bit h of j removed); the side s flips by w's bit h
                                    r = (C.flags & 1u) ? walsh_lev<8>(vi, C.lev) : walsh_lev<8>(vr, C.lev);
                                    if (ps.s & (C.flags >> 2)) r = -r;
                                } else {
                                    r = (C.flags & 1u) ? walsh_lev<16>(vi, C.lev) : walsh_lev<16>(vr, C.lev);
                                }
                                const uint32_t neg = ((uint32_t)__popcll(rep & C.z) ^ (uint32_t)__popc(threadIdx.x & C.tz) ^
                                                      (C.flags >> 1)) & 1u;
                                c[k] = neg ? -r * fac : r * fac;
                            }
                        }
                        const float red = warp_sum4<float>(c[0], c[1], c[2], c[3]);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (lane == 8 * k && q0 + k < G.s_end) acc[(q0 + k - a.s_begin) * nwarps + warp] += red;
                    }
                    continue;
                }
                if (use_x && K >= kXformMinStrings) {
                    // both parts from one sweep over the partners
                    float vr[16], vi[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const Cx<R> u = own[j];
                        if (G.X) {
                            const Cx<R> w = t[(threadIdx.x + j * 512u) ^ G.X];
                            vr[j] = w.x * u.x + w.y * u.y;
                            vi[j] = w.x * u.y - w.y * u.x;
                        } else {
                            vr[j] = u.x * u.x + u.y * u.y;
                            vi[j] = 0.f;
                        }
                    }
                    for (int part_i = 0; part_i < 2; ++part_i) {
                        if (!((G.parts >> part_i) & 1)) continue;   // no string uses this part
                        xform_part(part_i ? vi : vr, scr, lsg);
                        __syncthreads();
                        for (int q = G.s_begin + (int)threadIdx.x; q < G.s_end; q += 512) {
                            const DevString S = strs[q];
                            if ((S.nY & 1) != part_i) continue;
                            const uint32_t tau = (uint32_t)(S.z & ((1ull << a.kl) - 1ull)) |
                                                 ((S.bz & ((1u << tc.ash) - 1u)) << a.kl);
                            float c = xform_coef(scr, (S.bz >> tc.ash) & 15u, tau >> 5, tau & 31u);
                            const int neg = (__popcll(rep & S.z) ^ (G.X ? ((S.nY == 1) | (S.nY == 2)) : 0)) & 1;
                            acc[(q - a.s_begin) * nwarps] += neg ? -c : c;
                        }
                        __syncthreads();
                    }
                    continue;
                }
            }
            int ifac = 1;
            const uint32_t sel = G.X ? pair_select(tc, G.X, a.kl, EPT, ifac) : 0xFFFFFFFFu;
            const R fac = (R)ifac;
            for (int cs = G.s_begin; cs < G.s_end; cs += kEvcChunk) {
                const int nc = min(kEvcChunk, G.s_end - cs);
                uint32_t jm[kEvcChunk];
                int base[kEvcChunk], odd[kEvcChunk];
                R accr[kEvcChunk];
#pragma unroll
                for (int s = 0; s < kEvcChunk; ++s) {
                    const DevString S = strs[cs + (s < nc ? s : 0)];
                    jm[s] = walsh_mask(S.bz >> tc.ash);
                    odd[s] = S.nY & 1;
                    const int neg0 = G.X ? ((S.nY == 1) | (S.nY == 2)) : 0;
                    base[s] = (__popcll((rep | tc.l) & S.z) ^ __popc(tc.a0 & S.bz) ^ neg0) & 1;
                    accr[s] = 0;
                }
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const uint32_t e = threadIdx.x + j * blockDim.x;
                    if (e >= E || !((sel >> j) & 1u)) continue;
                    const Cx<R> u = own[j];
                    R wr, wi;
                    if (G.X) {
                        const Cx<R> v = t[e ^ G.X];
                        wr = v.x * u.x + v.y * u.y;    // Re(conj(v) u)
                        wi = v.x * u.y - v.y * u.x;    // Im(conj(v) u)
                    } else {
                        wr = u.x * u.x + u.y * u.y;    // |psi|^2 (x = 0, nY = 0)
                        wi = 0;
                    }
#pragma unroll
                    for (int s = 0; s < kEvcChunk; ++s) {
                        if (s < nc) {
                            const R val = odd[s] ? wi : wr;
                            accr[s] += ((base[s] ^ (jm[s] >> j)) & 1u) ? -val : val;
                        }
                    }
                }
#pragma unroll
                for (int s = 0; s < kEvcChunk; ++s) {
                    if (s < nc) {
                        const R v = warp_sum<R>(accr[s] * fac);
                        if (lane == 0) acc[(cs + s - a.s_begin) * nwarps + warp] += v;
                    }
                }
            }
        }
        __syncthreads();
        if (it + 2 < mine) load_coset<R>(t, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
        if constexpr (sizeof(R) == 4) {
            // the next writes to the slots follow the next coset's barrier
            if (((it + 1) % kEvcFlush) == 0 || it + 1 == mine) {
                for (int q = threadIdx.x; q < nslots; q += blockDim.x) {
                    float f = 0.f;
                    for (int w = 0; w < nwarps; ++w) {
                        f += acc[q * nwarps + w];
                        acc[q * nwarps + w] = 0.f;
                    }
                    tot64[q] += (double)f;
                }
            }
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
        double tsum = 0.0;
        if constexpr (sizeof(R) == 4) tsum = tot64[s];
        else
            for (int w = 0; w < nwarps; ++w) tsum += acc[s * nwarps + w];
        part[(size_t)blockIdx.x * part_stride + a.s_begin + s] = tsum;
    }
}

// K-EVC, few-string passes (every group one string, at most kEvcFew groups --
// the case of random Pauli strings): the per-thread pair split and sign data
// are computed once per kernel; per coset each group adds its FP32 partial
// into a per-thread shared-memory slot (the state's real type), flushed into
// FP64 registers every 64 cosets; one FP64 reduction at the end.

template <typename R, int EPT, bool ODD>
__device__ __forceinline__ R evc_pairs(const Cx<R> *t, const Cx<R> *own, uint32_t X, uint32_t sel, int base,
                                       uint32_t jm, uint32_t E) {
    R acc = 0;
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const uint32_t e = threadIdx.x + j * blockDim.x;
        if (e >= E || !((sel >> j) & 1u)) continue;
        const Cx<R> u = own[j], v = t[e ^ X];
        const R val = ODD ? (v.x * u.y - v.y * u.x) : (v.x * u.x + v.y * u.y);
        acc += ((base ^ (jm >> j)) & 1u) ? -val : val;
    }
    return acc;
}

template <typename R, int EPT, int LOGNT>
__global__ void __launch_bounds__(1 << LOGNT, 1) k_evc_few(const Cx<R> *__restrict__ psi, const CosetArgs a,
                                                    const DevGroup *__restrict__ groups,
                                                    const DevString *__restrict__ strs, double *__restrict__ part,
                                                    int part_stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    const int ng = a.g_end - a.g_begin;          // == number of strings (one per group)
    const int NT = blockDim.x;
    Cx<R> *buf = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(buf + 2 * E);
    R *acc32 = reinterpret_cast<R *>(spanv + (1u << a.m));             // [ng][NT], the state's real type
    uint32_t *pg = reinterpret_cast<uint32_t *>(acc32 + kEvcFew * NT);  // [ng][NT]: sel | code << 16 | tconst << 31
    __shared__ uint64_t gz[kEvcFew];
    __shared__ uint32_t gX[kEvcFew], gjm[kEvcFew], gw[kEvcFew];
    __shared__ int gmeta[kEvcFew];                                      // odd | fac << 1
    __shared__ double wsum[kEvcFew][32];                                // FP64 per string and warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < kEvcFew * 32; j += NT) wsum[j / 32][j % 32] = 0.0;
    coset_span(a, spanv);
    const ThreadCoset tc = thread_coset(a.kl);
    uint32_t tmask = 0;                                                 // bit g: sign constant of group g
    for (int g = 0; g < ng; ++g) {
        const DevGroup G = groups[a.g_begin + g];
        const DevString S = strs[G.s_begin];
        int fac = 1;
        const uint32_t sel = G.X ? pair_select(tc, G.X, a.kl, EPT, fac) : 0xFFFFu;
        const int neg0 = G.X ? ((S.nY == 1) | (S.nY == 2)) : 0;
        const int tconst = (__popcll(tc.l & S.z) ^ __popc(tc.a0 & S.bz) ^ neg0) & 1;
        const PairSel ps = G.X ? pair_split(tc, G.X, a.kl, EPT) : PairSel{-1, 0, 1};
        // packed: sel (bits 0..15), fast-path code (h + 1) | s << 3 | odd << 4
        // (bits 16..20, h + 1 = 0: every element), sign constant (bit 31)
        const uint32_t code = (uint32_t)(ps.h + 1) | ((uint32_t)ps.s << 3) | ((uint32_t)(S.nY & 1) << 4);
        pg[g * NT + threadIdx.x] = (sel & 0xFFFFu) | (code << 16) | ((uint32_t)tconst << 31);
        tmask |= (uint32_t)tconst << g;
        acc32[g * NT + threadIdx.x] = (R)0;
        if (threadIdx.x == 0) {
            gz[g] = S.z;
            gX[g] = G.X;
            gjm[g] = walsh_mask(S.bz >> tc.ash);
            gw[g] = S.bz >> tc.ash;
            gmeta[g] = (S.nY & 1) | (fac << 1);
        }
    }
    __syncthreads();
    const uint64_t ncos = 1ull << a.nfree;
    const uint64_t mine = blockIdx.x < ncos ? (ncos - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const bool fast = (NT == (1 << LOGNT)) && (E == ((uint32_t)EPT << LOGNT)) && EPT >= 2;
    // coset representatives walked with masked additions: rep_cur of the
    // current iteration, rep_pf of the one two ahead (the next copy issued)
    const BitWalk bw = bit_walk(a.freeb, a.nfree, gridDim.x);
    uint64_t rep_pf = deposit(blockIdx.x, a.freeb, a.nfree), rep_cur = rep_pf;
    for (uint64_t k = 0; k < 2; ++k) {
        if (k < mine) load_coset<R>(buf + k * E, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t rep = rep_cur;
        rep_cur = walk_next(rep_cur, bw);
        Cx<R> *t = buf + (it & 1) * E;
        cp_async_wait1();
        __syncthreads();
        Cx<R> own[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = threadIdx.x + j * blockDim.x;
            own[j] = e < E ? t[e] : mk<R>(0, 0);
        }
        // bit g: parity(rep & z_g) of every group at once (lane g computes it)
        const uint32_t bmask =
            tmask ^ __ballot_sync(0xffffffffu, lane < ng && ((__popcll(rep & gz[lane < ng ? lane : 0]) & 1) != 0));
        for (int g = 0; g < ng; ++g) {
            const uint32_t p = pg[g * NT + threadIdx.x];
            const uint32_t X = gX[g];
            const int meta = gmeta[g];
            const int base = (bmask >> g) & 1;
            const uint32_t sel = X ? (p & 0xFFFFu) : 0xFFFFFFFFu;
            R v;
            if (fast) {
                v = evc_fast<R, EPT, LOGNT>(t, own, X, (p >> 16) & 31u, gw[g]);
                if (base) v = -v;
            } else if (X == 0u) {
                v = 0;
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const uint32_t e = threadIdx.x + j * blockDim.x;
                    if (e >= E) continue;
                    const R q = own[j].x * own[j].x + own[j].y * own[j].y;
                    v += ((base ^ (gjm[g] >> j)) & 1u) ? -q : q;
                }
            } else if (meta & 1) {
                v = evc_pairs<R, EPT, true>(t, own, X, sel, base, gjm[g], E);
            } else {
                v = evc_pairs<R, EPT, false>(t, own, X, sel, base, gjm[g], E);
            }
            acc32[g * NT + threadIdx.x] += v;
        }
        if ((it & 63) == 63 || it + 1 == mine) {
            // flush: FP64 warp sums (times the pair factor) into the per-warp slots (fixed order)
            for (int g = 0; g < ng; ++g) {
                double v = (double)acc32[g * NT + threadIdx.x] * (double)(gmeta[g] >> 1);
                acc32[g * NT + threadIdx.x] = (R)0;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) wsum[g][warp] += v;
            }
        }
        __syncthreads();
        if (it + 2 < mine) load_coset<R>(t, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    __syncthreads();
    if (threadIdx.x < ng) {
        double tsum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += wsum[threadIdx.x][w];
        part[(size_t)blockIdx.x * part_stride + a.s_begin + threadIdx.x] = tsum;
    }
}

// ---- K-EVC few-string pass, three-stage ring --------------------------
// The pass of k_evc_few's fast layout (512 threads, EPT elements each, E =
// 512 EPT) with every per-group constant set once per launch: per thread the
// partner base address of the pair split (side included), the fold code and
// the constant part of the sign; per group (shared) the signs of the element
// Walsh fold per level.  Cosets stream through three shared buffers, so the
// copies of coset it + 2 are issued right after the one barrier of iteration
// it and two cosets are in flight while one is evaluated.

template <typename R> struct LevT { R s[4]; };

// sum over the selected elements (bit H of j equal to S; j' = j with bit H
// removed) of the pair term, folded by the level signs
template <typename R, int EPT, int SH, int H, int S, bool ODD>
__device__ __forceinline__ R evc_sel2(uint32_t sb, const Cx<R> *own, uint32_t B, const LevT<R> &lv) {
    constexpr int N = EPT / 2;
    R val[N];
#pragma unroll
    for (int jp = 0; jp < N; ++jp) {
        const int j0 = ((jp >> H) << (H + 1)) | (jp & ((1 << H) - 1));
        const Cx<R> u = own[j0 | (S << H)];
        const Cx<R> v = lds_cx<R>(sb + (B ^ ((uint32_t)j0 << SH)));
        val[jp] = ODD ? (v.x * u.y - v.y * u.x) : (v.x * u.x + v.y * u.y);
    }
#pragma unroll
    for (int i = 0, n = N; n > 1; ++i, n >>= 1) {
#pragma unroll
        for (int k = 0; k < n / 2; ++k) val[k] = fma(lv.s[i], val[2 * k + 1], val[2 * k]);
    }
    return val[0];
}
// every element (no split; X = 0 gives |own|^2)
template <typename R, int EPT, int SH, bool ODD>
__device__ __forceinline__ R evc_all2(uint32_t sb, const Cx<R> *own, uint32_t B, bool diag, const LevT<R> &lv) {
    R val[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const Cx<R> u = own[j];
        if (diag) {
            val[j] = u.x * u.x + u.y * u.y;
        } else {
            const Cx<R> v = lds_cx<R>(sb + (B ^ ((uint32_t)j << SH)));
            val[j] = ODD ? (v.x * u.y - v.y * u.x) : (v.x * u.x + v.y * u.y);
        }
    }
#pragma unroll
    for (int i = 0, n = EPT; n > 1; ++i, n >>= 1) {
#pragma unroll
        for (int k = 0; k < n / 2; ++k) val[k] = fma(lv.s[i], val[2 * k + 1], val[2 * k]);
    }
    return val[0];
}

// complex64 forms of evc_sel2 / evc_all2 on packed f32x2 registers: the
// products (v.x u.x, v.y u.y) -- or, with the partner's halves swapped on
// load, (v.y u.x, v.x u.y) for the imaginary part -- and the level folds run
// on both halves at once; the halves are combined at the end
__device__ __forceinline__ unsigned long long lds_b64(uint32_t addr) {
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ unsigned long long lds_b64_swap(uint32_t addr) {
    float x, y;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(addr));
    return f2_pack(y, x);
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
struct LevP { unsigned long long s[4]; };
template <bool ODD> __device__ __forceinline__ float f2_combine(unsigned long long r) {
    const float2 h = f2_unpack(r);
    return ODD ? h.y - h.x : h.x + h.y;
}
template <int EPT, int SH, int H, int S, bool ODD>
__device__ __forceinline__ float evc_sel2p(uint32_t sb, const unsigned long long *own, uint32_t B, const LevP &lv) {
    constexpr int N = EPT / 2;
    unsigned long long val[N];
#pragma unroll
    for (int jp = 0; jp < N; ++jp) {
        const int j0 = ((jp >> H) << (H + 1)) | (jp & ((1 << H) - 1));
        const uint32_t ad = sb + (B ^ ((uint32_t)j0 << SH));
        val[jp] = f2_mul(ODD ? lds_b64_swap(ad) : lds_b64(ad), own[j0 | (S << H)]);
    }
#pragma unroll
    for (int i = 0, n = N; n > 1; ++i, n >>= 1) {
#pragma unroll
        for (int k = 0; k < n / 2; ++k) val[k] = f2_fma(lv.s[i], val[2 * k + 1], val[2 * k]);
    }
    return f2_combine<ODD>(val[0]);
}
template <int EPT, int SH, bool ODD>
__device__ __forceinline__ float evc_all2p(uint32_t sb, const unsigned long long *own, uint32_t B, bool diag,
                                           const LevP &lv) {
    unsigned long long val[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        if (diag) {
            val[j] = f2_mul(own[j], own[j]);
        } else {
            const uint32_t ad = sb + (B ^ ((uint32_t)j << SH));
            val[j] = f2_mul(ODD ? lds_b64_swap(ad) : lds_b64(ad), own[j]);
        }
    }
#pragma unroll
    for (int i = 0, n = EPT; n > 1; ++i, n >>= 1) {
#pragma unroll
        for (int k = 0; k < n / 2; ++k) val[k] = f2_fma(lv.s[i], val[2 * k + 1], val[2 * k]);
    }
    return f2_combine<ODD>(val[0]);
}

// Coset copy of the ring's layout (E = NT EPT, 16-byte chunks, 2^kl-element
// runs with kl small enough that a thread's chunks share their position
// inside a run): chunk i of thread t is element c = t P + NT P i, P per
// chunk; its span index (c >> kl) = c0 + i step and run offset c & lowmask
// are per-thread constants, so each chunk costs one span load and an xor.
struct RingLoad {
    uint32_t s0, step;
    uint64_t low;
};
template <typename R, int NT>
__device__ __forceinline__ RingLoad ring_load_setup(int kl) {
    constexpr uint32_t P = 16 / sizeof(Cx<R>);
    const uint32_t c = threadIdx.x * P;
    return {c >> kl, ((uint32_t)NT * P) >> kl, (uint64_t)(c & ((1u << kl) - 1u))};
}
template <typename R, int EPT, int NT>
__device__ __forceinline__ void ring_load(Cx<R> *dst, const Cx<R> *psi, uint64_t rep, const uint64_t *spanv,
                                          const RingLoad &L) {
    constexpr uint32_t P = 16 / sizeof(Cx<R>);
    const uint64_t rc = rep ^ L.low;
    const uint64_t *sp = spanv + L.s0;
    Cx<R> *d = dst + threadIdx.x * P;
#pragma unroll
    for (int i = 0; i < EPT / (int)P; ++i) cp_async16(d + NT * P * i, psi + (rc ^ sp[i * L.step]));
}

template <typename R, int EPT, int LOGNT>
__global__ void __launch_bounds__(1 << LOGNT, 1) k_evc_ring(const Cx<R> *__restrict__ psi, const CosetArgs a,
                                                            const DevGroup *__restrict__ groups,
                                                            const DevString *__restrict__ strs,
                                                            double *__restrict__ part, int part_stride) {
    constexpr int NT = 1 << LOGNT;
    constexpr int SH = LOGNT + (sizeof(R) == 4 ? 3 : 4);   // byte offset of element row j: j << SH
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    const int ng = a.g_end - a.g_begin;          // == number of strings (one per group), at most kEvcFew
    Cx<R> *buf = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(buf + 3 * (size_t)E);
    __shared__ LevT<R> glev[kEvcFew];
    __shared__ LevP glevp[kEvcFew];                 // complex64: the level signs packed (s, s)
    __shared__ uint64_t gz[kEvcFew];
    __shared__ R gfac[kEvcFew];
    __shared__ double wsum[kEvcFew][NT / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < kEvcFew * (NT / 32); j += NT) wsum[j / (NT / 32)][j % (NT / 32)] = 0.0;
    coset_span(a, spanv);
    const ThreadCoset tc = thread_coset(a.kl);
    // per group: packed per-thread constants (partner base | code << 20 | sign bit 31)
    uint32_t pk[kEvcFew];
    uint32_t tmask = 0;
#pragma unroll
    for (int g = 0; g < kEvcFew; ++g) {
        pk[g] = 0;
        if (g < ng) {
            const DevGroup G = groups[a.g_begin + g];
            const DevString S = strs[G.s_begin];
            const uint32_t w = S.bz >> tc.ash;
            const PairSel ps = G.X ? pair_split(tc, G.X, a.kl, EPT) : PairSel{-1, 0, 1};
            uint32_t wf = w, flip = 0;
            if (ps.h >= 0) {
                wf = (w & ((1u << ps.h) - 1u)) | ((w >> (ps.h + 1)) << ps.h);
                flip = (uint32_t)ps.s & (w >> ps.h) & 1u;
            }
            const uint32_t neg0 = G.X ? (uint32_t)((S.nY == 1) | (S.nY == 2)) : 0u;
            const uint32_t tconst = ((uint32_t)__popc(tc.l & (uint32_t)S.z) ^ (uint32_t)__popc(tc.a0 & S.bz) ^ neg0 ^
                                     flip) & 1u;
            uint32_t B = (threadIdx.x ^ G.X) * (uint32_t)sizeof(Cx<R>);
            if (ps.h >= 0) B ^= (uint32_t)ps.s << (ps.h + SH);
            const uint32_t code = G.X ? ((uint32_t)(ps.h + 1) | ((uint32_t)ps.s << 3) | ((uint32_t)(S.nY & 1) << 4))
                                      : 31u;   // 31: the diagonal group
            pk[g] = B | (code << 20);
            tmask |= tconst << g;
            if (threadIdx.x == 0) {
                LevT<R> lv;
#pragma unroll
                for (int i = 0; i < 4; ++i) lv.s[i] = ((wf >> i) & 1u) ? (R)-1 : (R)1;
                glev[g] = lv;
                if constexpr (sizeof(R) == 4) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) glevp[g].s[i] = f2_pack((float)lv.s[i], (float)lv.s[i]);
                }
                gz[g] = S.z;
                gfac[g] = (R)ps.fac;
            }
        }
    }
    __syncthreads();
    const uint64_t ncos = 1ull << a.nfree;
    const uint64_t mine = blockIdx.x < ncos ? (ncos - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const BitWalk bw = bit_walk(a.freeb, a.nfree, gridDim.x);
    uint64_t rep_pf = deposit(blockIdx.x, a.freeb, a.nfree), rep_cur = rep_pf;
    // per-thread copy constants when a thread's chunks share their run offset
    const bool rl = a.kl <= LOGNT + (sizeof(R) == 4 ? 1 : 0) && (16u >> a.kl) <= (uint32_t)sizeof(Cx<R>) &&
                    (EPT * sizeof(Cx<R>)) % 16 == 0;
    const RingLoad RL = ring_load_setup<R, NT>(rl ? a.kl : 0);
    for (uint64_t k = 0; k < 2; ++k) {
        if (k < mine) {
            if (rl) ring_load<R, EPT, NT>(buf + k * E, psi, rep_pf, spanv, RL);
            else load_coset<R>(buf + k * E, psi, rep_pf, spanv, a.kl, E);
        }
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    R acc[kEvcFew];
#pragma unroll
    for (int g = 0; g < kEvcFew; ++g) acc[g] = 0;
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t rep = rep_cur;
        rep_cur = walk_next(rep_cur, bw);
        cp_async_wait1();
        __syncthreads();
        // coset it + 2 into the buffer of coset it - 1 (every thread is past it)
        if (it + 2 < mine) {
            if (rl) ring_load<R, EPT, NT>(buf + ((it + 2) % 3) * E, psi, rep_pf, spanv, RL);
            else load_coset<R>(buf + ((it + 2) % 3) * E, psi, rep_pf, spanv, a.kl, E);
        }
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
        const Cx<R> *t = buf + (it % 3) * E;
        const uint32_t sb = smem_u32(t);
        const uint32_t bmask =
            tmask ^ __ballot_sync(0xffffffffu, lane < ng && ((__popcll(rep & gz[lane < ng ? lane : 0]) & 1) != 0));
        if constexpr (sizeof(R) == 4) {
            unsigned long long own[EPT];
#pragma unroll
            for (int j = 0; j < EPT; ++j) own[j] = lds_b64(sb + ((threadIdx.x + j * NT) << 3));
#pragma unroll
            for (int g = 0; g < kEvcFew; ++g) {
                if (g < ng) {
                    const uint32_t B = pk[g] & 0xFFFFFu, code = pk[g] >> 20;
                    const LevP lv = glevp[g];
                    float v;
                    switch (code) {
                    case 0: v = evc_all2p<EPT, SH, false>(sb, own, B, false, lv); break;
                    case 16: v = evc_all2p<EPT, SH, true>(sb, own, B, false, lv); break;
                    case 31: v = evc_all2p<EPT, SH, false>(sb, own, B, true, lv); break;
#define SV_SEL2P(HH, SS, OO)                                                                                 \
    case (HH + 1) | (SS << 3) | (OO << 4):                                                                   \
        if constexpr ((2 << HH) <= EPT) v = evc_sel2p<EPT, SH, HH, SS, OO != 0>(sb, own, B, lv);             \
        else v = 0;                                                                                          \
        break;
#define SV_SEL2P_4(HH) SV_SEL2P(HH, 0, 0) SV_SEL2P(HH, 1, 0) SV_SEL2P(HH, 0, 1) SV_SEL2P(HH, 1, 1)
                        SV_SEL2P_4(0) SV_SEL2P_4(1) SV_SEL2P_4(2) SV_SEL2P_4(3)
#undef SV_SEL2P_4
#undef SV_SEL2P
                    default: v = 0; break;
                    }
                    acc[g] += ((bmask >> g) & 1u) ? -v : v;
                }
            }
        } else {
        Cx<R> own[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) own[j] = t[threadIdx.x + j * NT];
#pragma unroll
        for (int g = 0; g < kEvcFew; ++g) {
            if (g < ng) {
                const uint32_t B = pk[g] & 0xFFFFFu, code = pk[g] >> 20;
                const LevT<R> lv = glev[g];
                R v;
                switch (code) {
                case 0: v = evc_all2<R, EPT, SH, false>(sb, own, B, false, lv); break;
                case 16: v = evc_all2<R, EPT, SH, true>(sb, own, B, false, lv); break;
                case 31: v = evc_all2<R, EPT, SH, false>(sb, own, B, true, lv); break;
#define SV_SEL2(HH, SS, OO)                                                                                  \
    case (HH + 1) | (SS << 3) | (OO << 4):                                                                   \
        if constexpr ((2 << HH) <= EPT) v = evc_sel2<R, EPT, SH, HH, SS, OO != 0>(sb, own, B, lv);           \
        else v = 0;                                                                                          \
        break;
#define SV_SEL2_4(HH) SV_SEL2(HH, 0, 0) SV_SEL2(HH, 1, 0) SV_SEL2(HH, 0, 1) SV_SEL2(HH, 1, 1)
                    SV_SEL2_4(0) SV_SEL2_4(1) SV_SEL2_4(2) SV_SEL2_4(3)
#undef SV_SEL2_4
#undef SV_SEL2
                default: v = 0; break;
                }
                acc[g] += ((bmask >> g) & 1u) ? -v : v;
            }
        }
        }
        if ((it & 63) == 63 || it + 1 == mine) {
            // flush: FP64 warp sums (times the pair factor) into the per-warp slots (fixed order)
#pragma unroll
            for (int g = 0; g < kEvcFew; ++g) {
                if (g < ng) {
                    double v = (double)acc[g] * (double)gfac[g];
                    acc[g] = 0;
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) wsum[g][warp] += v;
                }
            }
        }
    }
    cp_async_wait0();
    __syncthreads();
    if (threadIdx.x < ng) {
        double tsum = 0.0;
        for (int w = 0; w < NT / 32; ++w) tsum += wsum[threadIdx.x][w];
        part[(size_t)blockIdx.x * part_stride + a.s_begin + threadIdx.x] = tsum;
    }
}

// ------------------------------------------------------------------ K-HPSI --
// lambda[b] += sum_t a_t i^nY (-1)^{|(b^x)&z|} psi[b^x] for every group of the
// pass (P|c> = i^nY (-1)^{|c&z|} |c^x>, c = b^x; parity((b^x)&z) =
// parity(b&z) ^ (nY & 1)).  The first pass stores, later passes add (the old
// lambda is loaded into registers while the coset is processed); the last
// pass also accumulates Re<psi|lambda>.  Same thread mapping and sign
// factorisation as K-EVC.
template <typename R, int EPT, bool ODD>
__device__ __forceinline__ void hpsi_one(Cx<R> *acc, const Cx<R> *t, uint32_t X, int base, uint32_t jm, R g,
                                         uint32_t E) {
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const uint32_t e = threadIdx.x + j * blockDim.x;
        if (e >= E) continue;
        const Cx<R> v = t[e ^ X];
        const R f = ((base ^ (jm >> j)) & 1u) ? -g : g;
        if (ODD) {            // i * v
            acc[j].x -= f * v.y;
            acc[j].y += f * v.x;
        } else {
            acc[j].x += f * v.x;
            acc[j].y += f * v.y;
        }
    }
}

// Fast path of hpsi_one (NT = 512, E = EPT * 512): compile-time element
// offsets, the sign as a bit flip of the coefficient.
template <typename R, int EPT, bool ODD>
__device__ __forceinline__ void hpsi_fast(Cx<R> *acc, const Cx<R> *t, uint32_t X, uint32_t sm, R g) {
    const uint32_t xl = X & 511u, xh = X >> 9;
    const Cx<R> *tb = t + (threadIdx.x ^ xl);
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const Cx<R> v = tb[((uint32_t)j ^ xh) << 9];
        R f;
        switch (j) {
#define SV_FB(J) case J: f = flip_bit<J>(g, sm); break;
            SV_FB(0) SV_FB(1) SV_FB(2) SV_FB(3) SV_FB(4) SV_FB(5) SV_FB(6) SV_FB(7)
            SV_FB(8) SV_FB(9) SV_FB(10) SV_FB(11) SV_FB(12) SV_FB(13) SV_FB(14) SV_FB(15)
#undef SV_FB
        default: f = g; break;
        }
        if (ODD) {
            acc[j].x -= f * v.y;
            acc[j].y += f * v.x;
        } else {
            acc[j].x += f * v.x;
            acc[j].y += f * v.y;
        }
    }
}

// complex64, 16 amplitudes per thread (NT = 512, E = 8192): the signed
// coefficient of element j is built along a Gray chain written out (each
// one XOR from an earlier one), and the partner of element j is at byte
// offset B ^ (j << 12) of the staged coset (B = (t ^ X) * 8) whose shared
// address is sb.
template <bool ODD>
__device__ __forceinline__ void hpsi_gray16(float2 *acc, uint32_t sb, uint32_t B, uint32_t g0, uint32_t w) {
    const uint32_t F0 = (w & 1u) << 31, F1 = (w & 2u) << 30, F2 = (w & 4u) << 29, F3 = (w & 8u) << 28;
    const uint32_t g1 = g0 ^ F0, g2 = g0 ^ F1, g3 = g2 ^ F0, g4 = g0 ^ F2, g5 = g4 ^ F0, g6 = g4 ^ F1,
                   g7 = g6 ^ F0, g8 = g0 ^ F3, g9 = g8 ^ F0, g10 = g8 ^ F1, g11 = g10 ^ F0, g12 = g8 ^ F2,
                   g13 = g12 ^ F0, g14 = g12 ^ F1, g15 = g14 ^ F0;
#define SV_HG(J)                                                                                 \
    {                                                                                            \
        const float2 v = lds_cx<float>(sb + (B ^ ((uint32_t)(J) << 12)));                        \
        const float f = __uint_as_float(g##J);                                                   \
        if (ODD) {                                                                               \
            acc[J].x = fmaf(-f, v.y, acc[J].x);                                                  \
            acc[J].y = fmaf(f, v.x, acc[J].y);                                                   \
        } else {                                                                                 \
            acc[J].x = fmaf(f, v.x, acc[J].x);                                                   \
            acc[J].y = fmaf(f, v.y, acc[J].y);                                                   \
        }                                                                                        \
    }
    SV_HG(0) SV_HG(1) SV_HG(2) SV_HG(3) SV_HG(4) SV_HG(5) SV_HG(6) SV_HG(7)
    SV_HG(8) SV_HG(9) SV_HG(10) SV_HG(11) SV_HG(12) SV_HG(13) SV_HG(14) SV_HG(15)
#undef SV_HG
}

// hpsi_gray16 with the partner's row offset XH = (X >> 9) fixed at compile
// time: the partner of element j is at Bl + ((j ^ XH) << 12), Bl = shared
// address of the coset + (t ^ (X & 511)) * 8, so every load is one register
// plus an immediate (rows 8..15 from Bl + 32 KiB, keeping immediates small).
template <bool ODD, int XH>
__device__ __forceinline__ void hpsi_row16(float2 *acc, uint32_t Bl, uint32_t g0, uint32_t w) {
    const uint32_t Bh = Bl + 32768u;
    const uint32_t F0 = (w & 1u) << 31, F1 = (w & 2u) << 30, F2 = (w & 4u) << 29, F3 = (w & 8u) << 28;
    const uint32_t g1 = g0 ^ F0, g2 = g0 ^ F1, g3 = g2 ^ F0, g4 = g0 ^ F2, g5 = g4 ^ F0, g6 = g4 ^ F1,
                   g7 = g6 ^ F0, g8 = g0 ^ F3, g9 = g8 ^ F0, g10 = g8 ^ F1, g11 = g10 ^ F0, g12 = g8 ^ F2,
                   g13 = g12 ^ F0, g14 = g12 ^ F1, g15 = g14 ^ F0;
#define SV_HR(J)                                                                                 \
    {                                                                                            \
        const float2 v = (((J) ^ XH) < 8) ? lds_f2_off<(((J) ^ XH) & 7) << 12>(Bl)               \
                                          : lds_f2_off<(((J) ^ XH) & 7) << 12>(Bh);              \
        const float f = __uint_as_float(g##J);                                                   \
        if (ODD) {                                                                               \
            acc[J].x = fmaf(-f, v.y, acc[J].x);                                                  \
            acc[J].y = fmaf(f, v.x, acc[J].y);                                                   \
        } else {                                                                                 \
            acc[J].x = fmaf(f, v.x, acc[J].x);                                                   \
            acc[J].y = fmaf(f, v.y, acc[J].y);                                                   \
        }                                                                                        \
    }
    SV_HR(0) SV_HR(1) SV_HR(2) SV_HR(3) SV_HR(4) SV_HR(5) SV_HR(6) SV_HR(7)
    SV_HR(8) SV_HR(9) SV_HR(10) SV_HR(11) SV_HR(12) SV_HR(13) SV_HR(14) SV_HR(15)
#undef SV_HR
}

// Strings of one H|psi> pass staged once per launch (complex64, 16 amplitudes
// per thread, 512 threads, at most kHpsiTab strings): per string the signed
// coefficient, X (bit 31: nY odd), w and z; per thread the coset-independent
// sign bits parity(l & z) ^ parity(a0 & bz) ^ nY of every string.  Per coset
// one ballot gives parity(rep & z) of every string.
constexpr int kHpsiTab = 32;
struct HpsiTab {
    uint64_t z[kHpsiTab];
    uint32_t X[kHpsiTab], g[kHpsiTab], w[kHpsiTab];
};

__device__ __forceinline__ void hpsi_tab_string(float2 *acc, const HpsiTab &T, int k, uint32_t sb, uint32_t bmask) {
    const uint32_t Xo = T.X[k];
    const uint32_t g0 = T.g[k] ^ (((bmask >> k) & 1u) << 31);
    const uint32_t w = T.w[k];
    const uint32_t Bl = sb + ((threadIdx.x ^ (Xo & 511u)) << 3);
    switch (((Xo >> 9) & 15u) | ((Xo >> 31) << 4)) {
#define SV_HC(C) case C: hpsi_row16<((C) >> 4) != 0, (C) & 15>(acc, Bl, g0, w); break;
        SV_HC(0) SV_HC(1) SV_HC(2) SV_HC(3) SV_HC(4) SV_HC(5) SV_HC(6) SV_HC(7)
        SV_HC(8) SV_HC(9) SV_HC(10) SV_HC(11) SV_HC(12) SV_HC(13) SV_HC(14) SV_HC(15)
        SV_HC(16) SV_HC(17) SV_HC(18) SV_HC(19) SV_HC(20) SV_HC(21) SV_HC(22) SV_HC(23)
        SV_HC(24) SV_HC(25) SV_HC(26) SV_HC(27) SV_HC(28) SV_HC(29) SV_HC(30) SV_HC(31)
#undef SV_HC
    default: break;
    }
}

template <typename R, int EPT>
__global__ void __launch_bounds__(512, 1) k_hpsi_pass(const Cx<R> *__restrict__ psi, Cx<R> *__restrict__ lam,
                                                      const CosetArgs a, const DevGroup *__restrict__ groups,
                                                      const DevString *__restrict__ strs, int first, int last,
                                                      double *__restrict__ epart, int *status, long long limit) {
    (void)status; (void)limit;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    Cx<R> *buf = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(buf + 2 * E);
    __shared__ double wsum[32];
    coset_span(a, spanv);
    const ThreadCoset tc = thread_coset(a.kl);
    const uint32_t lowmask = (1u << a.kl) - 1u;
    const uint64_t ncos = 1ull << a.nfree;
    const uint64_t mine = blockIdx.x < ncos ? (ncos - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const bool fast = (blockDim.x == 512) && (E == (uint32_t)EPT * 512u);
    // coset representatives walked with masked additions: rep_cur of the
    // current iteration, rep_pf of the one two ahead (the next copy issued)
    const BitWalk bw = bit_walk(a.freeb, a.nfree, gridDim.x);
    uint64_t rep_pf = deposit(blockIdx.x, a.freeb, a.nfree), rep_cur = rep_pf;
    for (uint64_t k = 0; k < 2; ++k) {
        if (k < mine) load_coset<R>(buf + k * E, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    // string table (complex64, 16 per thread, 512 threads, few strings)
    __shared__ HpsiTab tabs;
    int ns = 0;
    uint32_t tmask = 0;
    if constexpr (sizeof(R) == 4 && EPT == 16) {
        if (fast) {
            for (int gi = a.g_begin; gi < a.g_end; ++gi) {
                const DevGroup G = groups[gi];
                for (int sidx = G.s_begin; sidx < G.s_end; ++sidx, ++ns) {
                    if (ns >= kHpsiTab) continue;
                    const DevString S = strs[sidx];
                    tmask |= (uint32_t)((__popcll(tc.l & S.z) ^ __popc(tc.a0 & S.bz) ^ S.nY) & 1) << ns;
                    if (threadIdx.x == 0) {
                        const float g = (S.nY & 2) ? -(float)S.coef : (float)S.coef;
                        tabs.z[ns] = S.z;
                        tabs.X[ns] = G.X | ((uint32_t)(S.nY & 1) << 31);
                        tabs.g[ns] = __float_as_uint(g);
                        tabs.w[ns] = S.bz >> tc.ash;
                    }
                }
            }
            __syncthreads();
        }
    }
    const bool tabbed = ns > 0 && ns <= kHpsiTab;
    const int lane = threadIdx.x & 31;
    double eacc = 0.0;
    R eblk = 0;
    for (uint64_t it = 0; it < mine; ++it) {
        const uint64_t rep = rep_cur;
        rep_cur = walk_next(rep_cur, bw);
        Cx<R> *t = buf + (it & 1) * E;
        Cx<R> acc[EPT], old[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = threadIdx.x + j * blockDim.x;
            acc[j] = mk<R>(0, 0);
            old[j] = mk<R>(0, 0);
            if (!first && e < E) old[j] = lam[rep ^ spanv[e >> a.kl] ^ (e & lowmask)];
        }
        cp_async_wait1();
        __syncthreads();
        if constexpr (sizeof(R) == 4 && EPT == 16) {
            if (tabbed) {
                const bool pb = lane < ns && ((__popcll(rep & tabs.z[lane < ns ? lane : 0]) & 1) != 0);
                const uint32_t bmask = tmask ^ __ballot_sync(0xffffffffu, pb);
                const uint32_t sb = smem_u32(t);
                for (int k = 0; k < ns; ++k)
                    hpsi_tab_string(reinterpret_cast<float2 *>(acc), tabs, k, sb, bmask);
            }
        }
        for (int gi = tabbed ? a.g_end : a.g_begin; gi < a.g_end; ++gi) {
            const DevGroup G = groups[gi];
            for (int s = G.s_begin; s < G.s_end; ++s) {
                const DevString S = strs[s];
                const int base = (__popcll((rep | tc.l) & S.z) ^ __popc(tc.a0 & S.bz) ^ S.nY) & 1;
                const R g = (S.nY & 2) ? -(R)S.coef : (R)S.coef;
                if constexpr (sizeof(R) == 4 && EPT == 16) {
                    if (fast) {
                        const uint32_t g0 = __float_as_uint((float)g) ^ ((uint32_t)base << 31);
                        const uint32_t B = (threadIdx.x ^ G.X) * 8u;
                        if (S.nY & 1) hpsi_gray16<true>(reinterpret_cast<float2 *>(acc), smem_u32(t), B, g0, S.bz >> tc.ash);
                        else hpsi_gray16<false>(reinterpret_cast<float2 *>(acc), smem_u32(t), B, g0, S.bz >> tc.ash);
                        continue;
                    }
                }
                const uint32_t jm = walsh_mask(S.bz >> tc.ash);
                if (fast) {
                    const uint32_t sm = base ? ~jm : jm;
                    if (S.nY & 1) hpsi_fast<R, EPT, true>(acc, t, G.X, sm, g);
                    else hpsi_fast<R, EPT, false>(acc, t, G.X, sm, g);
                } else if (S.nY & 1) {
                    hpsi_one<R, EPT, true>(acc, t, G.X, base, jm, g, E);
                } else {
                    hpsi_one<R, EPT, false>(acc, t, G.X, base, jm, g, E);
                }
            }
        }
        R eloc = 0;
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = threadIdx.x + j * blockDim.x;
            if (e >= E) continue;
            acc[j].x += old[j].x;
            acc[j].y += old[j].y;
            lam[rep ^ spanv[e >> a.kl] ^ (e & lowmask)] = acc[j];
            if (last) {
                const Cx<R> p = t[e];
                eloc += p.x * acc[j].x + p.y * acc[j].y;
            }
        }
        if (last) {
            // FP32 over up to 64 cosets, then FP64 (1/64 of the FP32 rate here)
            eblk += eloc;
            if (((it + 1) & 63) == 0) {
                eacc += (double)eblk;
                eblk = 0;
            }
        }
        __syncthreads();
        if (it + 2 < mine) load_coset<R>(t, psi, rep_pf, spanv, a.kl, E);
        cp_async_commit();
        rep_pf = walk_next(rep_pf, bw);
    }
    if (last) {
        double v = eacc + (double)eblk;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += wsum[w];
            epart[blockIdx.x] = tsum;
        }
    }
}

// ----------------------------------------------------------------- K-BATCH --
// Many independent small states in ONE persistent launch.  A CTA takes a whole
// state at a time from an atomic work counter (states pre-sorted longest
// first) and runs, on its own workspace: |psi> = |init>, the QSU gate passes
// of the state's plan (no virtual chunks), lambda = H psi by the coset passes
// of the shared Hamiltonian with the energy Re<psi|lambda>, and the adjoint
// reverse sweep with per-gate gradient partials (FP64 sums at the end).  No CTA ever waits for
// another CTA; every barrier is a __syncthreads inside one CTA.  Per-state
// start/end device times (globaltimer, ns) give the latency distribution.


__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Register-phased tile of a gate pass inside the batched kernel (512
// threads): the tile is staged swizzled, each phase gathers the thread's
// 2^RB amplitudes, applies its gates in registers, scatters them back.
template <typename R, int RB>
__device__ __noinline__ void batch_reg_forward(Cx<R> *tile, const GatePassArgs &P, const DevOp *ops, const Phase *phases,
                                  const R *coef) {
    constexpr int V = 1 << RB;
    for (int ph = P.ph_begin; ph < P.ph_end; ++ph) {
        const Phase F = phases[ph];
        uint32_t base, sp[V];
        phase_index<RB>(F.rmask, P.k, base, sp);
        base = phase_base(F.rmask, F.lanes, P.k);   // the phase's lane bits (conflict-free half-warps)
        Cx<R> x[V];
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = tile[swz_tile(base | sp[v])];
        for (int o = F.op_begin; o < F.op_end; ++o) reg_apply<R, RB>(x, ops[o], F.rmask, base, coef, nullptr, false);
#pragma unroll
        for (int v = 0; v < V; ++v) tile[swz_tile(base | sp[v])] = x[v];
        __syncthreads();
    }
}

// psi and lambda tiles of a register-phased reverse pass staged swizzled,
// with all of a thread's V loads of both in flight before its first store
template <typename R, int V>
__device__ __noinline__ void batch_load_pair(Cx<R> *tp, Cx<R> *tl, const Cx<R> *psi, const Cx<R> *lam, uint64_t base,
                                             const uint64_t *hioff, int nlow) {
    const uint32_t lowmask = (1u << nlow) - 1u;
    Cx<R> vp[V], vl[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t j = threadIdx.x + (uint32_t)v * blockDim.x;
        const uint64_t gi = base | hioff[j >> nlow] | (j & lowmask);
        vp[v] = psi[gi];
        vl[v] = lam[gi];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t j = threadIdx.x + (uint32_t)v * blockDim.x;
        tp[swz_tile(j)] = vp[v];
        tl[swz_tile(j)] = vl[v];
    }
}

template <typename R, int RB>
__device__ __noinline__ void batch_reg_adjoint(Cx<R> *tp, Cx<R> *tl, const GatePassArgs &P, const DevOp *ops,
                                  const Phase *phases, const R *coef, R *opacc, int o0) {
    constexpr int V = 1 << RB;
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ph = P.ph_end - 1; ph >= P.ph_begin; --ph) {
        const Phase F = phases[ph];
        uint32_t base, sp[V];
        phase_index<RB>(F.rmask, P.k, base, sp);
        base = phase_base(F.rmask, F.lanes, P.k);   // the phase's lane bits (conflict-free half-warps)
        Cx<R> xp[V], xl[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t si = swz_tile(base | sp[v]);
            xp[v] = tp[si];
            xl[v] = tl[si];
        }
        for (int o = F.op_end - 1; o >= F.op_begin; --o) {
            const DevOp op = ops[o];
            R g = reg_adjoint<R, RB>(xp, xl, op, F.rmask, base, coef, nullptr);
            if (has_param(op.kind)) {
                g = warp_sum<R>(g);
                if (lane == 0) opacc[(o - o0) * nwarps + warp] += g;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t si = swz_tile(base | sp[v]);
            tp[si] = xp[v];
            tl[si] = xl[v];
        }
        __syncthreads();
    }
}

constexpr int kBatchMaxOps = 512;      // gate operations per state (smem accumulators)
constexpr int kBatchMaxGates = 1024;

template <typename R, int EPT>
__global__ void __launch_bounds__(512, 1) k_batch(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int NT = blockDim.x, nwarps = NT >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t TILE = 1u << a.kmax;                              // staged amplitudes per buffer
    Cx<R> *tp = reinterpret_cast<Cx<R> *>(smem);
    Cx<R> *tl = tp + TILE;
    uint64_t *hioff = reinterpret_cast<uint64_t *>(tl + TILE);       // 2^hio entries (>= 2^(k - nlow), >= 256)
    // per op and warp a gradient partial of the state's real type over the
    // state's tiles (FP64 is 1/64 of the FP32 rate here), summed in FP64 at the end
    unsigned char *opbase = reinterpret_cast<unsigned char *>(hioff + (1u << a.hio));
    R *opacc = reinterpret_cast<R *>(opbase);                                        // [kBatchMaxOps][nwarps]
    R *coef = reinterpret_cast<R *>(opbase + (size_t)kBatchMaxOps * nwarps * 8);     // [2 * kBatchMaxGates]
    __shared__ int s_state;
    __shared__ double s_red[32];
    __shared__ HpsiTab tabs;
    const size_t N = (size_t)1 << a.n;
    Cx<R> *psi = reinterpret_cast<Cx<R> *>(a.work) + (size_t)blockIdx.x * 2 * N;
    Cx<R> *lam = psi + N;
    while (true) {
        if (threadIdx.x == 0) s_state = atomicAdd(a.counter, 1);
        __syncthreads();
        const int si = s_state;
        if (si >= a.nstates) break;
        const int st = a.order[si];
        const unsigned long long t0 = globaltimer_ns();
        const int plan = a.state_plan[st];
        const int g0 = a.gate_off[st], ng = a.gate_off[st + 1] - g0;
        const int p0 = a.param_off[st], np = a.param_off[st + 1] - p0;
        const int o0 = a.plan_op_off[plan], nops = a.plan_op_off[plan + 1] - o0;
        for (int g = threadIdx.x; g < ng; g += NT) {
            const int p = a.gparam[g0 + g];
            double c = 1.0, sn = 0.0;
            if (p >= 0) sincos(0.5 * a.params[p0 + p], &sn, &c);
            coef[2 * g] = (R)c;
            coef[2 * g + 1] = (R)sn;
        }
        for (int j = threadIdx.x; j < nops * nwarps; j += NT) opacc[j] = 0;
        for (size_t i = threadIdx.x; i < N; i += NT) psi[i] = mk<R>(i == a.init_index ? 1 : 0, 0);
        __syncthreads();
        // ---- QSU
        for (int pi = a.plan_pass_off[plan]; pi < a.plan_pass_off[plan + 1]; ++pi) {
            const GatePassArgs &P = a.passes[pi];
            const uint32_t T = 1u << P.k, nh = 1u << (P.k - P.nlow), lowmask = (1u << P.nlow) - 1u;
            for (uint32_t j = threadIdx.x; j < nh; j += NT) hioff[j] = deposit(j, P.hi, P.nhi);
            __syncthreads();
            const int rb = (P.ph_begin >= 0 && NT == 512) ? P.k - 9 : 0;   // register-phased pass
            const uint64_t ntl = 1ull << P.nout;
            if (rb >= 2 && rb <= 4) {
                // tiles alternate between the two buffers; the next one streams in
                load_tile_async<R>(tp, psi, deposit(0, P.out, P.nout), hioff, P.nlow, T);
                cp_async_commit();
                for (uint64_t ti = 0; ti < ntl; ++ti) {
                    const uint64_t base = deposit(ti, P.out, P.nout);
                    Cx<R> *cur = (ti & 1) ? tl : tp;
                    if (ti + 1 < ntl)
                        load_tile_async<R>((ti & 1) ? tp : tl, psi, deposit(ti + 1, P.out, P.nout), hioff, P.nlow, T);
                    cp_async_commit();
                    cp_async_wait1();
                    __syncthreads();
                    if (rb == 4) batch_reg_forward<R, 4>(cur, P, a.ops, a.phases, coef);
                    else if (rb == 3) batch_reg_forward<R, 3>(cur, P, a.ops, a.phases, coef);
                    else batch_reg_forward<R, 2>(cur, P, a.ops, a.phases, coef);
                    for (uint32_t j = threadIdx.x; j < T; j += NT)
                        psi[base | hioff[j >> P.nlow] | (j & lowmask)] = cur[swz_tile(j)];
                    __syncthreads();
                }
                continue;
            }
            for (uint64_t ti = 0; ti < ntl; ++ti) {
                const uint64_t base = deposit(ti, P.out, P.nout);
                for (uint32_t j = threadIdx.x; j < T; j += NT) tp[j] = psi[base | hioff[j >> P.nlow] | (j & lowmask)];
                __syncthreads();
                for (int o = P.op_begin; o < P.op_end; ++o) {
                    const DevOp op = a.ops[o];
                    apply_op<R>(tp, P.k, op, coef, nullptr, false);
                    __syncthreads();
                }
                for (uint32_t j = threadIdx.x; j < T; j += NT) psi[base | hioff[j >> P.nlow] | (j & lowmask)] = tp[j];
                __syncthreads();
            }
        }
        // ---- lambda = H psi, energy
        double eacc = 0.0;
        for (int hp = 0; hp < a.nhpass; ++hp) {
            const CosetArgs &C = a.hpass[hp];
            const uint32_t E = 1u << (C.kl + C.m), M = 1u << C.m, lm = (1u << C.kl) - 1u;
            uint64_t *spanv = hioff;                     // M <= 256 entries
            for (uint32_t j = threadIdx.x; j < M; j += NT) {
                uint64_t v = 0;
                for (int i = 0; i < C.m; ++i)
                    if (j >> i & 1u) v ^= C.basis[i];
                spanv[j] = v;
            }
            const ThreadCoset tc = thread_coset(C.kl);
            const uint64_t ncos = 1ull << C.nfree;
            const bool fast = (NT == 512) && (E == (uint32_t)EPT * 512u);
            // the pass's strings staged once (as in k_hpsi_pass); the table of
            // the previous pass is no longer read (barrier at its end)
            int ns = 0;
            uint32_t tmask = 0;
            if constexpr (sizeof(R) == 4 && EPT == 16) {
                if (fast) {
                    for (int gi = C.g_begin; gi < C.g_end; ++gi) {
                        const DevGroup G = a.groups[gi];
                        for (int sidx = G.s_begin; sidx < G.s_end; ++sidx, ++ns) {
                            if (ns >= kHpsiTab) continue;
                            const DevString S = a.strs[sidx];
                            tmask |= (uint32_t)((__popcll(tc.l & S.z) ^ __popc(tc.a0 & S.bz) ^ S.nY) & 1) << ns;
                            if (threadIdx.x == 0) {
                                const float gf = (S.nY & 2) ? -(float)S.coef : (float)S.coef;
                                tabs.z[ns] = S.z;
                                tabs.X[ns] = G.X | ((uint32_t)(S.nY & 1) << 31);
                                tabs.g[ns] = __float_as_uint(gf);
                                tabs.w[ns] = S.bz >> tc.ash;
                            }
                        }
                    }
                }
            }
            const bool tabbed = ns > 0 && ns <= kHpsiTab;
            __syncthreads();
            // cosets alternate between the two buffers (lambda's buffer is free
            // here); the next one streams in while the current one is used
            load_coset<R>(tp, psi, deposit(0, C.freeb, C.nfree), spanv, C.kl, E);
            cp_async_commit();
            for (uint64_t ci = 0; ci < ncos; ++ci) {
                const uint64_t rep = deposit(ci, C.freeb, C.nfree);
                Cx<R> *cur = (ci & 1) ? tl : tp;
                if (ci + 1 < ncos) load_coset<R>((ci & 1) ? tp : tl, psi, deposit(ci + 1, C.freeb, C.nfree), spanv, C.kl, E);
                cp_async_commit();
                Cx<R> acc[EPT];
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const uint32_t e = threadIdx.x + j * NT;
                    acc[j] = mk<R>(0, 0);
                    if (hp > 0 && e < E) acc[j] = lam[rep ^ spanv[e >> C.kl] ^ (e & lm)];
                }
                cp_async_wait1();
                __syncthreads();
                if constexpr (sizeof(R) == 4 && EPT == 16) {
                    if (tabbed) {
                        const bool pb = lane < ns && ((__popcll(rep & tabs.z[lane < ns ? lane : 0]) & 1) != 0);
                        const uint32_t bmask = tmask ^ __ballot_sync(0xffffffffu, pb);
                        const uint32_t sb = smem_u32(cur);
                        for (int k = 0; k < ns; ++k)
                            hpsi_tab_string(reinterpret_cast<float2 *>(acc), tabs, k, sb, bmask);
                    }
                }
                for (int gi = tabbed ? C.g_end : C.g_begin; gi < C.g_end; ++gi) {
                    const DevGroup G = a.groups[gi];
                    for (int s = G.s_begin; s < G.s_end; ++s) {
                        const DevString S = a.strs[s];
                        const int base = (__popcll((rep | tc.l) & S.z) ^ __popc(tc.a0 & S.bz) ^ S.nY) & 1;
                        const R g = (S.nY & 2) ? -(R)S.coef : (R)S.coef;
                        if constexpr (sizeof(R) == 4 && EPT == 16) {
                            if (fast) {
                                const uint32_t g0 = __float_as_uint((float)g) ^ ((uint32_t)base << 31);
                                const uint32_t B = (threadIdx.x ^ G.X) * 8u;
                                const uint32_t sb = smem_u32(cur);
                                if (S.nY & 1)
                                    hpsi_gray16<true>(reinterpret_cast<float2 *>(acc), sb, B, g0, S.bz >> tc.ash);
                                else
                                    hpsi_gray16<false>(reinterpret_cast<float2 *>(acc), sb, B, g0, S.bz >> tc.ash);
                                continue;
                            }
                        }
                        const uint32_t jm = walsh_mask(S.bz >> tc.ash);
                        if (fast) {
                            const uint32_t sm = base ? ~jm : jm;
                            if (S.nY & 1) hpsi_fast<R, EPT, true>(acc, cur, G.X, sm, g);
                            else hpsi_fast<R, EPT, false>(acc, cur, G.X, sm, g);
                        } else if (S.nY & 1) {
                            hpsi_one<R, EPT, true>(acc, cur, G.X, base, jm, g, E);
                        } else {
                            hpsi_one<R, EPT, false>(acc, cur, G.X, base, jm, g, E);
                        }
                    }
                }
                R el = 0;
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const uint32_t e = threadIdx.x + j * NT;
                    if (e >= E) continue;
                    lam[rep ^ spanv[e >> C.kl] ^ (e & lm)] = acc[j];
                    el += cur[e].x * acc[j].x + cur[e].y * acc[j].y;
                }
                if (hp == a.nhpass - 1) eacc += (double)el;
                __syncthreads();
            }
        }
        if (a.nhpass == 0)
            for (size_t i = threadIdx.x; i < N; i += NT) lam[i] = mk<R>(0, 0);
        for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
        if (lane == 0) s_red[warp] = eacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double e = 0.0;
            for (int w = 0; w < nwarps; ++w) e += s_red[w];
            a.energies[st] = e;
        }
        // ---- adjoint reverse sweep
        for (int pi = a.plan_pass_off[plan + 1] - 1; pi >= a.plan_pass_off[plan]; --pi) {
            const GatePassArgs &P = a.passes[pi];
            const uint32_t T = 1u << P.k, nh = 1u << (P.k - P.nlow), lowmask = (1u << P.nlow) - 1u;
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < nh; j += NT) hioff[j] = deposit(j, P.hi, P.nhi);
            __syncthreads();
            const int rb = (P.ph_begin >= 0 && NT == 512) ? P.k - 9 : 0;   // register-phased pass
            for (uint64_t ti = 0; ti < (1ull << P.nout); ++ti) {
                const uint64_t base = deposit(ti, P.out, P.nout);
                if (rb >= 2 && rb <= 4) {
                    // T = 2^rb x 512 here
                    if (rb == 4) batch_load_pair<R, 16>(tp, tl, psi, lam, base, hioff, P.nlow);
                    else if (rb == 3) batch_load_pair<R, 8>(tp, tl, psi, lam, base, hioff, P.nlow);
                    else batch_load_pair<R, 4>(tp, tl, psi, lam, base, hioff, P.nlow);
                    __syncthreads();
                    if (rb == 4) batch_reg_adjoint<R, 4>(tp, tl, P, a.ops, a.phases, coef, opacc, o0);
                    else if (rb == 3) batch_reg_adjoint<R, 3>(tp, tl, P, a.ops, a.phases, coef, opacc, o0);
                    else batch_reg_adjoint<R, 2>(tp, tl, P, a.ops, a.phases, coef, opacc, o0);
                    for (uint32_t j = threadIdx.x; j < T; j += NT) {
                        const uint64_t gi = base | hioff[j >> P.nlow] | (j & lowmask);
                        psi[gi] = tp[swz_tile(j)];
                        lam[gi] = tl[swz_tile(j)];
                    }
                    __syncthreads();
                    continue;
                }
                for (uint32_t j = threadIdx.x; j < T; j += NT) {
                    const uint64_t gi = base | hioff[j >> P.nlow] | (j & lowmask);
                    tp[j] = psi[gi];
                    tl[j] = lam[gi];
                }
                __syncthreads();
                for (int o = P.op_end - 1; o >= P.op_begin; --o) {
                    const DevOp op = a.ops[o];
                    R g = adjoint_op<R>(tp, tl, P.k, op, coef, nullptr);
                    if (has_param(op.kind)) {
                        g = warp_sum<R>(g);
                        if (lane == 0) opacc[(o - o0) * nwarps + warp] += g;
                    }
                    __syncthreads();
                }
                for (uint32_t j = threadIdx.x; j < T; j += NT) {
                    const uint64_t gi = base | hioff[j >> P.nlow] | (j & lowmask);
                    psi[gi] = tp[j];
                    lam[gi] = tl[j];
                }
                __syncthreads();
            }
        }
        // gradient: per op, then per parameter in a fixed order
        if (threadIdx.x == 0) {
            for (int p = 0; p < np; ++p) a.grads[p0 + p] = 0.0;
            for (int o = 0; o < nops; ++o) {
                const DevOp op = a.ops[o0 + o];
                const int p = a.gparam[g0 + op.gate];
                if (p < 0 || !has_param(op.kind)) continue;
                double v = 0.0;
                for (int w = 0; w < nwarps; ++w) v += (double)opacc[o * nwarps + w];
                a.grads[p0 + p] += v;
            }
            a.t_start[st] = t0;
            a.t_end[st] = globaltimer_ns();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- Alg. 6 search --
// One greedy step of Alg. 6 on the device: every global set G (an nG-subset
// of the n qubits, by lexicographic rank r) counts the remaining strings
// whose X/Y support avoids G (weights = multiplicities); the step takes the
// largest count, ties to the smallest rank -- the first maximum in
// lexicographic order, as the host search does.  best = max over
// (count << 32) | (0xFFFFFFFF - r).
__global__ void k_alg6_step(const uint64_t *__restrict__ xs, const int32_t *__restrict__ w, int nx, int n, int k,
                            const int64_t *__restrict__ binom, uint64_t ncand, unsigned long long *best) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sx = reinterpret_cast<uint64_t *>(smem);
    int32_t *sw = reinterpret_cast<int32_t *>(sx + nx);
    int64_t *sb = reinterpret_cast<int64_t *>(sw + nx + (nx & 1));   // [(n + 1) * (k + 1)]: C(a, b)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        sx[i] = xs[i];
        sw[i] = w[i];
    }
    for (int i = threadIdx.x; i < (n + 1) * (k + 1); i += blockDim.x) sb[i] = binom[i];
    __syncthreads();
    unsigned long long mine = 0;
    for (uint64_t r0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r0 < ncand; r0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t G = 0;
        int64_t r = (int64_t)r0;
        int c = 0;
        for (int i = 0; i < k; ++i) {
            while (true) {
                const int a = n - c - 1, b = k - i - 1;
                const int64_t cnt = (a >= 0 && b <= a) ? sb[a * (k + 1) + b] : 0;
                if (r < cnt) break;
                r -= cnt;
                ++c;
            }
            G |= 1ull << c;
            ++c;
        }
        unsigned int cnt = 0;
        for (int i = 0; i < nx; ++i) cnt += (sx[i] & G) ? 0u : (unsigned int)sw[i];
        const unsigned long long key = ((unsigned long long)cnt << 32) | (0xFFFFFFFFull - r0);
        mine = key > mine ? key : mine;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, mine, o);
        mine = other > mine ? other : mine;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, mine);
}

// ------------------------------------------------------------ small kernels --
template <typename R>
__global__ void k_prep(const int32_t *__restrict__ gparam, const double *__restrict__ params, int m,
                       R *__restrict__ coef) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= m) return;
    const int p = gparam[g];
    double c = 1.0, s = 0.0;
    if (p >= 0) sincos(0.5 * params[p], &s, &c);
    coef[2 * g] = (R)c;
    coef[2 * g + 1] = (R)s;
}

template <typename R>
__global__ void k_set_one(Cx<R> *psi, uint64_t index) {
    psi[index] = mk<R>(1, 0);
}

__global__ void k_reduce_rows(const double *__restrict__ part, int nblocks, int stride, int s_begin, int s_end,
                              double *__restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int s = s_begin + w;
    if (s >= s_end) return;
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) acc += part[(size_t)b * stride + s];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[s] = acc;
}

__global__ void k_scatter(const double *__restrict__ opval, const int32_t *__restrict__ off,
                          const int32_t *__restrict__ idx, int np, double *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int i = off[p]; i < off[p + 1]; ++i) s += opval[idx[i]];
    grad[p] = s;
}

__global__ void k_energy(const double *__restrict__ slotval, const int32_t *__restrict__ term_slot,
                         const double *__restrict__ coeffs, int nterms, double *__restrict__ per_term,
                         double *__restrict__ energy) {
    __shared__ double red[256];
    double s = 0.0;
    for (int t = threadIdx.x; t < nterms; t += blockDim.x) {
        const double v = slotval[term_slot[t]];
        if (per_term) per_term[t] = v;
        s += coeffs[t] * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *energy = red[0];
}

template <typename R>
__global__ void k_copy(Cx<R> *__restrict__ dst, const Cx<R> *__restrict__ src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <typename K>
int occupancy(K kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) nb = 1;
    return nb < 1 ? 1 : nb;
}

// Largest dynamic shared memory a block may opt in to on the current device.
int smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
        v = 48 * 1024;
    return v;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t gate_smem(sv_dtype dt, int k, int nlow) {
    const size_t es = dt == SV_C64 ? 8 : 16;
    return ((size_t)1 << k) * es + ((size_t)1 << (k - nlow)) * 8 + 64;
}
size_t adj_smem(sv_dtype dt, int k, int nlow, int nops, int threads) {
    const size_t es = dt == SV_C64 ? 8 : 16;
    return 2 * ((size_t)1 << k) * es + ((size_t)1 << (k - nlow)) * 8 + (size_t)nops * (threads / 32) * 8 + 64;
}
size_t coset_smem(sv_dtype dt, int E, int m, int nslots, int nwarps) {
    const size_t rb = dt == SV_C64 ? 4 : 8;
    return evc_span_end((uint32_t)E, m, rb) + evc_slot_bytes(nslots, nwarps, rb);
}

}  // namespace

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int gate_pass_grid(sv_dtype dt, int k, int nlow, int nops, int threads, int blocks_per_sm) {
    (void)nops;
    size_t sm = gate_smem(dt, k, nlow);
    int nb;
    if (dt == SV_C64) { allow_smem(k_gate_pass<float>, sm); nb = occupancy(k_gate_pass<float>, threads, sm); }
    else { allow_smem(k_gate_pass<double>, sm); nb = occupancy(k_gate_pass<double>, threads, sm); }
    if (blocks_per_sm > 0) nb = std::min(nb, blocks_per_sm);
    return nb * device_sms();
}

int adj_pass_grid(sv_dtype dt, int k, int nlow, int nops, int threads, int blocks_per_sm) {
    size_t sm = adj_smem(dt, k, nlow, nops, threads);
    int nb;
    if (dt == SV_C64) { allow_smem(k_adj_pass<float>, sm); nb = occupancy(k_adj_pass<float>, threads, sm); }
    else { allow_smem(k_adj_pass<double>, sm); nb = occupancy(k_adj_pass<double>, threads, sm); }
    if (blocks_per_sm > 0) nb = std::min(nb, blocks_per_sm);
    return nb * device_sms();
}

int coset_grid(sv_dtype dt, int E, int blocks_per_sm, bool hpsi) {
    // one CTA per SM: each holds two staged cosets (double buffer); a fixed
    // grid per call so every pass writes the same partial rows
    (void)dt; (void)E; (void)hpsi;
    int per = 1;
    if (blocks_per_sm > 0) per = std::min(per, blocks_per_sm);
    return per * device_sms();
}

cudaError_t launch_prep(sv_dtype dt, cudaStream_t st, const int32_t *gparam, const double *params, int m,
                        void *coef) {
    if (m <= 0) return cudaSuccess;
    const int th = 128, bl = (m + th - 1) / th;
    if (dt == SV_C64) k_prep<float><<<bl, th, 0, st>>>(gparam, params, m, (float *)coef);
    else k_prep<double><<<bl, th, 0, st>>>(gparam, params, m, (double *)coef);
    return cudaGetLastError();
}

cudaError_t launch_set_basis(sv_dtype dt, cudaStream_t st, void *psi, size_t bytes, uint64_t index) {
    cudaError_t e = cudaMemsetAsync(psi, 0, bytes, st);
    if (e != cudaSuccess) return e;
    if (dt == SV_C64) k_set_one<float><<<1, 1, 0, st>>>((float2 *)psi, index);
    else k_set_one<double><<<1, 1, 0, st>>>((double2 *)psi, index);
    return cudaGetLastError();
}

cudaError_t launch_gate_pass(sv_dtype dt, cudaStream_t st, int grid, int threads, void *psi,
                             const GatePassArgs &a, const DevOp *ops, const void *coef, const void *mats) {
    size_t sm = gate_smem(dt, a.k, a.nlow);
    if (dt == SV_C64) {
        allow_smem(k_gate_pass<float>, sm);
        k_gate_pass<float><<<grid, threads, sm, st>>>((float2 *)psi, a, ops, (const float *)coef,
                                                      (const float2 *)mats);
    } else {
        allow_smem(k_gate_pass<double>, sm);
        k_gate_pass<double><<<grid, threads, sm, st>>>((double2 *)psi, a, ops, (const double *)coef,
                                                       (const double2 *)mats);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t gate_reg_dispatch(cudaStream_t st, int grid, void *psi, const GatePassArgs &a, const DevOp *ops,
                              const Phase *phases, const RegStep *steps, const void *coef, const void *mats,
                              const DiagBlock *dblocks, const DiagMember *dmem) {
    const size_t sm = gate_reg_smem(sizeof(R) == 4 ? SV_C64 : SV_C128, a);
    switch (a.k - 9) {
#define SV_GR(RB)                                                                                            \
    case RB:                                                                                                 \
        allow_smem(k_gate_reg<R, RB>, sm);                                                                   \
        k_gate_reg<R, RB><<<grid, kRegThreads, sm, st>>>((Cx<R> *)psi, a, ops, phases, steps, (const R *)coef, \
                                                         (const Cx<R> *)mats, dblocks, dmem);                \
        break;
        SV_GR(2) SV_GR(3)
    case 4:   // complex128 tiles hold at most 2^12 amplitudes
        if constexpr (sizeof(R) == 4) {
            allow_smem(k_gate_reg<R, 4>, sm);
            k_gate_reg<R, 4><<<grid, kRegThreads, sm, st>>>((Cx<R> *)psi, a, ops, phases, steps, (const R *)coef,
                                                            (const Cx<R> *)mats, dblocks, dmem);
            break;
        }
        return cudaErrorInvalidValue;
#undef SV_GR
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t adj_reg_dispatch(cudaStream_t st, int grid, void *psi, void *lam, const GatePassArgs &a,
                             const DevOp *ops, const Phase *phases, const RegStep *steps, const void *coef,
                             const void *mats, double *part, int part_stride, const DiagBlock *dblocks,
                             const DiagMember *dmem) {
    const size_t sm = adj_reg_smem(sizeof(R) == 4 ? SV_C64 : SV_C128, a);
    switch (a.k - 9) {
#define SV_AR(RB)                                                                                            \
    case RB:                                                                                                 \
        allow_smem(k_adj_reg<R, RB>, sm);                                                                    \
        k_adj_reg<R, RB><<<grid, kRegThreads, sm, st>>>((Cx<R> *)psi, (Cx<R> *)lam, a, ops, phases, steps,   \
                                                        (const R *)coef, (const Cx<R> *)mats, part, part_stride, \
                                                        dblocks, dmem);                                      \
        break;
        SV_AR(2) SV_AR(3)
    case 4:
        if constexpr (sizeof(R) == 4) {
            allow_smem(k_adj_reg<R, 4>, sm);
            k_adj_reg<R, 4><<<grid, kRegThreads, sm, st>>>((Cx<R> *)psi, (Cx<R> *)lam, a, ops, phases, steps,
                                                           (const R *)coef, (const Cx<R> *)mats, part, part_stride,
                                                           dblocks, dmem);
            break;
        }
        return cudaErrorInvalidValue;
#undef SV_AR
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t gate_reg_smem(sv_dtype dt, const GatePassArgs &a) {
    const int amp = dt == SV_C64 ? 8 : 16;
    return 2 * ((size_t)1 << a.k) * amp + reg_layout(a, amp, false).total;
}

size_t adj_reg_smem(sv_dtype dt, const GatePassArgs &a) {
    const int amp = dt == SV_C64 ? 8 : 16;
    return 2 * ((size_t)1 << a.k) * amp + reg_layout(a, amp, true).total;
}

cudaError_t launch_gate_reg(sv_dtype dt, cudaStream_t st, int grid, void *psi, const GatePassArgs &a,
                            const DevOp *ops, const Phase *phases, const RegStep *steps, const void *coef,
                            const void *mats, const DiagBlock *dblocks, const DiagMember *dmem) {
    if (dt == SV_C64) return gate_reg_dispatch<float>(st, grid, psi, a, ops, phases, steps, coef, mats, dblocks, dmem);
    return gate_reg_dispatch<double>(st, grid, psi, a, ops, phases, steps, coef, mats, dblocks, dmem);
}

cudaError_t launch_adj_reg(sv_dtype dt, cudaStream_t st, int grid, void *psi, void *lam, const GatePassArgs &a,
                           const DevOp *ops, const Phase *phases, const RegStep *steps, const void *coef,
                           const void *mats, double *part, int part_stride, const DiagBlock *dblocks,
                           const DiagMember *dmem) {
    if (dt == SV_C64)
        return adj_reg_dispatch<float>(st, grid, psi, lam, a, ops, phases, steps, coef, mats, part, part_stride,
                                       dblocks, dmem);
    return adj_reg_dispatch<double>(st, grid, psi, lam, a, ops, phases, steps, coef, mats, part, part_stride,
                                    dblocks, dmem);
}

cudaError_t launch_adj_pass(sv_dtype dt, cudaStream_t st, int grid, int threads, void *psi, void *lam,
                            const GatePassArgs &a, const DevOp *ops, const void *coef, const void *mats,
                            double *part, int part_stride) {
    size_t sm = adj_smem(dt, a.k, a.nlow, a.op_end - a.op_begin, threads);
    if (dt == SV_C64) {
        allow_smem(k_adj_pass<float>, sm);
        k_adj_pass<float><<<grid, threads, sm, st>>>((float2 *)psi, (float2 *)lam, a, ops, (const float *)coef,
                                                     (const float2 *)mats, part, part_stride);
    } else {
        allow_smem(k_adj_pass<double>, sm);
        k_adj_pass<double><<<grid, threads, sm, st>>>((double2 *)psi, (double2 *)lam, a, ops,
                                                      (const double *)coef, (const double2 *)mats, part,
                                                      part_stride);
    }
    return cudaGetLastError();
}

cudaError_t launch_bitswap(sv_dtype dt, cudaStream_t st, void *psi, int n, const int32_t *pairs, int npairs,
                           int blocks_per_sm) {
    if (npairs <= 0) return cudaSuccess;
    SwapArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    // tile = the longest low run L with L + (partners of paired run bits) <= TB
    const int TB = dt == SV_C64 ? 12 : 11;
    int L = std::min(n, TB);
    for (; L > 1; --L) {
        int partners = 0;
        for (int i = 0; i < npairs; ++i) {
            const int p = std::min(pairs[2 * i], pairs[2 * i + 1]), q = std::max(pairs[2 * i], pairs[2 * i + 1]);
            if (p < L && q >= L) ++partners;
        }
        if (L + partners <= TB) break;
    }
    a.L = L;
    int tb[24], ntb = 0;
    for (int i = 0; i < npairs; ++i) {
        const int p = std::min(pairs[2 * i], pairs[2 * i + 1]), q = std::max(pairs[2 * i], pairs[2 * i + 1]);
        if (q < a.L) {
            a.la[a.nlo] = (int8_t)p; a.lb[a.nlo] = (int8_t)q; ++a.nlo;
        } else if (p < a.L) {
            tb[ntb++] = q;
        } else {
            a.ha[a.nhi] = (int8_t)p; a.hb[a.nhi] = (int8_t)q; ++a.nhi;
        }
    }
    std::sort(tb, tb + ntb);
    for (int i = 0; i < ntb; ++i) a.tb[i] = (int8_t)tb[i];
    a.ntb = a.L + ntb;
    for (int i = 0; i < npairs; ++i) {
        const int p = std::min(pairs[2 * i], pairs[2 * i + 1]), q = std::max(pairs[2 * i], pairs[2 * i + 1]);
        if (p < a.L && q >= a.L) {
            const int r = (int)(std::lower_bound(tb, tb + ntb, q) - tb);
            a.la[a.nlo] = (int8_t)p; a.lb[a.nlo] = (int8_t)(a.L + r); ++a.nlo;
        }
    }
    uint64_t inside = (1ull << a.L) - 1;
    for (int i = 0; i < ntb; ++i) inside |= 1ull << tb[i];
    a.nout = 0;
    for (int b = 0; b < n; ++b)
        if (!(inside >> b & 1)) a.out[a.nout++] = (int8_t)b;
    const size_t es = dt == SV_C64 ? 8 : 16;
    const size_t sm = 2 * ((size_t)1 << a.ntb) * es + ((size_t)1 << (a.ntb - a.L)) * 8 + ((size_t)1 << a.ntb) * 2;
    const int threads = 256;
    int grid;
    if (dt == SV_C64) {
        allow_smem(k_bitswap<float>, sm);
        grid = occupancy(k_bitswap<float>, threads, sm);
    } else {
        allow_smem(k_bitswap<double>, sm);
        grid = occupancy(k_bitswap<double>, threads, sm);
    }
    if (blocks_per_sm > 0) grid = std::min(grid, blocks_per_sm);
    grid *= device_sms();
    const uint64_t ntiles = 1ull << a.nout;
    if ((uint64_t)grid > ntiles) grid = (int)ntiles;
    if (dt == SV_C64) k_bitswap<float><<<grid, threads, sm, st>>>((float2 *)psi, a);
    else k_bitswap<double><<<grid, threads, sm, st>>>((double2 *)psi, a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t evc_dispatch(cudaStream_t st, int grid, const void *psi, const CosetArgs &a, const DevGroup *groups,
                         const DevString *strs, double *part, int part_stride, int *status, long long limit) {
    const int E = 1 << (a.kl + a.m);
    // threads: a multiple of the run length, at least one warp, at most 512
    const int threads = std::max(std::max(32, 1 << a.kl), std::min(E, 512));
    const int ept = std::max(1, E / threads);
    const bool ring_fits = 3 * (size_t)E * sizeof(Cx<R>) + ((size_t)1 << a.m) * 8 + 4096 <= (size_t)smem_optin();
    if (a.few && threads == 512 && ept >= 2 && ept <= 16 && E == (uint32_t)ept * 512u && ring_fits) {
        const size_t smr = 3 * (size_t)E * sizeof(Cx<R>) + ((size_t)1 << a.m) * 8;
#define SV_EVCR_CASE(N)                                                                                      \
    case N:                                                                                                  \
        allow_smem(k_evc_ring<R, N, 9>, smr);                                                                \
        k_evc_ring<R, N, 9><<<grid, 512, smr, st>>>((const Cx<R> *)psi, a, groups, strs, part, part_stride); \
        return cudaGetLastError();
        switch (ept) {
            SV_EVCR_CASE(2)
            SV_EVCR_CASE(4)
            SV_EVCR_CASE(8)
            SV_EVCR_CASE(16)
        default:
            break;
        }
#undef SV_EVCR_CASE
    }
    if (a.few) {
        const size_t smf = 2 * (size_t)E * sizeof(Cx<R>) + ((size_t)1 << a.m) * 8 +
                           (size_t)kEvcFew * threads * (sizeof(R) + 4);
#define SV_EVCF_CASE(N)                                                                                      \
    case N:                                                                                                  \
        allow_smem(k_evc_few<R, N, 9>, smf);                                                                 \
        k_evc_few<R, N, 9><<<grid, threads, smf, st>>>((const Cx<R> *)psi, a, groups, strs, part,            \
                                                      part_stride);                                          \
        return cudaGetLastError();
        switch (ept) {
            SV_EVCF_CASE(1)
            SV_EVCF_CASE(2)
            SV_EVCF_CASE(4)
            SV_EVCF_CASE(8)
            SV_EVCF_CASE(16)
        default:
            return cudaErrorInvalidValue;
        }
#undef SV_EVCF_CASE
    }
    size_t sm = coset_smem(sizeof(R) == 4 ? SV_C64 : SV_C128, E, a.m, a.s_end - a.s_begin, threads / 32);
    // transform scratch for large groups (complex64, 16 per thread, 512 threads) when it fits
    int xform = 0;
    const size_t strc_bytes = (size_t)(a.s_end - a.s_begin) * sizeof(StrC);
    if (sizeof(R) == 4 && threads == 512 && E == 8192 && sm + kXformScratch * 4 + strc_bytes <= (size_t)smem_optin()) {
        sm += kXformScratch * 4 + strc_bytes;
        xform = 1;
    }
#define SV_EVC_CASE(N)                                                                                       \
    case N:                                                                                                  \
        allow_smem(k_evc_pass<R, N>, sm);                                                                    \
        k_evc_pass<R, N><<<grid, threads, sm, st>>>((const Cx<R> *)psi, a, groups, strs, part, part_stride, \
                                                    xform);                                                  \
        break;
    switch (ept) {
        SV_EVC_CASE(1)
        SV_EVC_CASE(2)
        SV_EVC_CASE(4)
        SV_EVC_CASE(8)
        SV_EVC_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SV_EVC_CASE
    return cudaGetLastError();
}

cudaError_t launch_evc_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, const CosetArgs &a,
                            const DevGroup *groups, const DevString *strs, double *part, int part_stride,
                            int *status, long long limit) {
    if (dt == SV_C64) return evc_dispatch<float>(st, grid, psi, a, groups, strs, part, part_stride, status, limit);
    return evc_dispatch<double>(st, grid, psi, a, groups, strs, part, part_stride, status, limit);
}

template <typename R>
cudaError_t hpsi_dispatch(cudaStream_t st, int grid, const void *psi, void *lam, const CosetArgs &a,
                          const DevGroup *groups, const DevString *strs, int first, int last, double *epart,
                          int *status, long long limit) {
    const int E = 1 << (a.kl + a.m);
    const size_t sm = 2 * (size_t)E * sizeof(Cx<R>) + ((size_t)1 << a.m) * 8;
    // a multiple of the run length, at least one warp, at most 512
    const int threads = std::max(std::max(32, 1 << a.kl), std::min(E, 512));
    const int ept = std::max(1, E / threads);
#define SV_HPSI_CASE(N)                                                                                      \
    case N:                                                                                                  \
        allow_smem(k_hpsi_pass<R, N>, sm);                                                                   \
        k_hpsi_pass<R, N><<<grid, threads, sm, st>>>((const Cx<R> *)psi, (Cx<R> *)lam, a, groups, strs,     \
                                                     first, last, epart, status, limit);                     \
        break;
    switch (ept) {
        SV_HPSI_CASE(1)
        SV_HPSI_CASE(2)
        SV_HPSI_CASE(4)
        SV_HPSI_CASE(8)
        SV_HPSI_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef SV_HPSI_CASE
    return cudaGetLastError();
}

cudaError_t launch_hpsi_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, void *lam,
                             const CosetArgs &a, const DevGroup *groups, const DevString *strs, int first,
                             int last, double *epart, int *status, long long limit) {
    if (dt == SV_C64) return hpsi_dispatch<float>(st, grid, psi, lam, a, groups, strs, first, last, epart, status, limit);
    return hpsi_dispatch<double>(st, grid, psi, lam, a, groups, strs, first, last, epart, status, limit);
}

cudaError_t launch_reduce_rows(cudaStream_t st, const double *part, int nblocks, int stride, int s_begin,
                               int s_end, double *out) {
    const int ns = s_end - s_begin;
    if (ns <= 0) return cudaSuccess;
    const int th = 256, warps_per = th / 32;
    const int bl = (ns + warps_per - 1) / warps_per;
    k_reduce_rows<<<bl, th, 0, st>>>(part, nblocks, stride, s_begin, s_end, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter(cudaStream_t st, const double *opval, const int32_t *off, const int32_t *idx, int np,
                           double *grad) {
    if (np <= 0) return cudaSuccess;
    k_scatter<<<(np + 127) / 128, 128, 0, st>>>(opval, off, idx, np, grad);
    return cudaGetLastError();
}

cudaError_t launch_energy(cudaStream_t st, const double *slotval, const int32_t *term_slot, const double *coeffs,
                          int nterms, double *per_term, double *energy) {
    k_energy<<<1, 256, 0, st>>>(slotval, term_slot, coeffs, nterms, per_term, energy);
    return cudaGetLastError();
}

cudaError_t launch_copy(sv_dtype dt, cudaStream_t st, void *dst, const void *src, size_t n) {
    const int th = 256;
    int bl = (int)std::min<size_t>((n + th - 1) / th, (size_t)device_sms() * 8);
    if (bl < 1) bl = 1;
    if (dt == SV_C64) k_copy<float><<<bl, th, 0, st>>>((float2 *)dst, (const float2 *)src, n);
    else k_copy<double><<<bl, th, 0, st>>>((double2 *)dst, (const double2 *)src, n);
    return cudaGetLastError();
}

size_t batch_smem(sv_dtype dt, int kmax, int hio, int threads) {
    const size_t es = dt == SV_C64 ? 8 : 16;
    return 2 * ((size_t)1 << kmax) * es + ((size_t)1 << hio) * 8 + (size_t)kBatchMaxOps * (threads / 32) * 8 +
           2 * (size_t)kBatchMaxGates * (es / 2);
}

int batch_max_ops() { return kBatchMaxOps; }
int batch_max_gates() { return kBatchMaxGates; }

// Instantiated kernels: each thread keeps EPT = 2^kmax / threads accumulators
// of an H|psi> coset pass in registers, EPT in {4, 8, 16}.
int batch_supported(sv_dtype dt, int kmax, int threads) {
    if (threads != 256 && threads != 512) return 0;
    if (kmax < 10 || kmax > (dt == SV_C64 ? 13 : 12)) return 0;
    const int ept = (1 << kmax) / threads;
    return ept == 4 || ept == 8 || ept == 16;
}

#define SV_BATCH_SWITCH(R, ept, ACTION) \
    switch (ept) {                        \
    case 4: ACTION(R, 4); break;          \
    case 8: ACTION(R, 8); break;          \
    default: ACTION(R, 16); break;        \
    }

int batch_occupancy(sv_dtype dt, int kmax, int hio, int threads) {
    if (!batch_supported(dt, kmax, threads)) return 0;
    const size_t sm = batch_smem(dt, kmax, hio, threads);
    const int ept = (1 << kmax) / threads;
    int occ = 0;
#define SV_BOCC(R, E)                       \
    allow_smem(k_batch<R, E>, sm);          \
    occ = occupancy(k_batch<R, E>, threads, sm);
    if (dt == SV_C64) { SV_BATCH_SWITCH(float, ept, SV_BOCC) }
    else { SV_BATCH_SWITCH(double, ept, SV_BOCC) }
#undef SV_BOCC
    return occ;
}

cudaError_t launch_batch(sv_dtype dt, cudaStream_t st, int grid, int threads, const BatchArgs &a) {
    if (!batch_supported(dt, a.kmax, threads)) return cudaErrorInvalidValue;
    const size_t sm = batch_smem(dt, a.kmax, a.hio, threads);
    const int ept = (1 << a.kmax) / threads;
    cudaError_t e = cudaSuccess;
#define SV_BLAUNCH(R, E)                                      \
    e = allow_smem(k_batch<R, E>, sm);                        \
    if (e == cudaSuccess) k_batch<R, E><<<grid, threads, sm, st>>>(a);
    if (dt == SV_C64) { SV_BATCH_SWITCH(float, ept, SV_BLAUNCH) }
    else { SV_BATCH_SWITCH(double, ept, SV_BLAUNCH) }
#undef SV_BLAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_alg6_step(cudaStream_t st, const uint64_t *xs, const int32_t *w, int nx, int n, int k,
                             const int64_t *binom, uint64_t ncand, unsigned long long *best) {
    const size_t sm = (size_t)nx * 8 + (size_t)(nx + (nx & 1)) * 4 + (size_t)(n + 1) * (k + 1) * 8;
    const int threads = 256;
    const uint64_t blocks = std::min<uint64_t>((ncand + threads - 1) / threads, (uint64_t)device_sms() * 8);
    cudaError_t e = cudaFuncSetAttribute(k_alg6_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_alg6_step<<<(int)std::max<uint64_t>(blocks, 1), threads, sm, st>>>(xs, w, nx, n, k, binom, ncand, best);
    return cudaGetLastError();
}

}  // namespace sv
