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

template <typename R>
__device__ __forceinline__ void rot(Cx<R> &u, Cx<R> &v, R c, R s) {
    const Cx<R> a = u, b = v;
    u = mk<R>(c * a.x - s * b.x, c * a.y - s * b.y);
    v = mk<R>(s * a.x + c * b.x, s * a.y + c * b.y);
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
    return kind == SV_RY || kind == SV_RZ || kind == SV_GIVENS || kind == SV_DEXC;
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
            const DevOp op = ops[o];
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
            const DevOp op = ops[o];
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
    for (uint32_t j = threadIdx.x; j < nh; j += blockDim.x) hioff[j] = deposit(j, a.tb, a.ntb - a.L);
    __syncthreads();
    const uint32_t runmask = (1u << a.L) - 1u;
    const uint64_t ntiles = 1ull << a.nout;
    const bool vec = (VEC == 2) && a.L >= 1;
    for (uint64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const uint64_t b0 = deposit(ti, a.out, a.nout);
        const uint64_t b1 = sigma_hi(b0, a);
        if (b1 < b0) continue;
        const bool self = (b1 == b0);
        if (self && a.nlo == 0) continue;
        if (vec) {
            for (uint32_t j = 2 * threadIdx.x; j < T; j += 2 * blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s = swz<R>(j);
                *reinterpret_cast<float4 *>(&A[s]) = *reinterpret_cast<const float4 *>(&psi[b0 | off]);
                if (!self) *reinterpret_cast<float4 *>(&B[s]) = *reinterpret_cast<const float4 *>(&psi[b1 | off]);
            }
        } else {
            for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s = swz<R>(j);
                A[s] = psi[b0 | off];
                if (!self) B[s] = psi[b1 | off];
            }
        }
        __syncthreads();
        if (vec) {
            for (uint32_t j = 2 * threadIdx.x; j < T; j += 2 * blockDim.x) {
                const uint64_t off = hioff[j >> a.L] | (j & runmask);
                const uint32_t s0 = swz<R>(sigma_lo(j, a)), s1 = swz<R>(sigma_lo(j + 1, a));
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
                const uint32_t s = swz<R>(sigma_lo(j, a));
                psi[b0 | off] = self ? A[s] : B[s];
                if (!self) psi[b1 | off] = A[s];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- K-EVC --
// For group x (X = its offset inside the staged coset) and each pair (b, b^x)
// with b's lowest X bit clear: w = conj(psi[b^x]) psi[b]; string (x, z) with
// nY = |x & z| adds  i^nY (-1)^{|b&z|} (w + (-1)^nY conj(w)), which is real:
//   nY = 0: +2 s Re w,  1: -2 s Im w,  2: -2 s Re w,  3: +2 s Im w,
// s = (-1)^{|b&z|} with b the FULL physical index (chunk bits included: the
// per-chunk sign s_j of Eq. par_exp).  x = 0 adds s |psi[b]|^2.
constexpr int kEvcChunk = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_evc_pass(const Cx<R> *__restrict__ psi, const CosetArgs a,
                                                  const DevGroup *__restrict__ groups,
                                                  const DevString *__restrict__ strs, double *__restrict__ part,
                                                  int part_stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    const uint32_t M = 1u << a.m;
    const int nslots = a.s_end - a.s_begin;
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Cx<R> *tile = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(tile + E);
    double *acc = reinterpret_cast<double *>(spanv + M);
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        uint64_t v = 0;
        for (int i = 0; i < a.m; ++i)
            if (j >> i & 1u) v ^= a.basis[i];
        spanv[j] = v;
    }
    for (int j = threadIdx.x; j < nslots * nwarps; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    const uint32_t lowmask = (1u << a.kl) - 1u;
    const uint64_t ncos = 1ull << a.nfree;
    for (uint64_t ci = blockIdx.x; ci < ncos; ci += gridDim.x) {
        const uint64_t rep = deposit(ci, a.freeb, a.nfree);
        for (uint32_t e = threadIdx.x; e < E; e += blockDim.x)
            tile[e] = psi[rep ^ spanv[e >> a.kl] ^ (e & lowmask)];
        __syncthreads();
        for (int gi = a.g_begin; gi < a.g_end; ++gi) {
            const DevGroup G = groups[gi];
            for (int cs = G.s_begin; cs < G.s_end; cs += kEvcChunk) {
                const int ns = min(kEvcChunk, G.s_end - cs);
                uint64_t z[kEvcChunk];
                int ny[kEvcChunk];
                R accr[kEvcChunk];
#pragma unroll
                for (int s = 0; s < kEvcChunk; ++s) {
                    z[s] = s < ns ? strs[cs + s].z : 0ull;
                    ny[s] = s < ns ? strs[cs + s].nY : 0;
                    accr[s] = 0;
                }
                if (G.X == 0u) {
                    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
                        const Cx<R> v = tile[e];
                        const R p = v.x * v.x + v.y * v.y;
                        const uint64_t b = rep ^ spanv[e >> a.kl] ^ (e & lowmask);
#pragma unroll
                        for (int s = 0; s < kEvcChunk; ++s)
                            accr[s] += (__popcll(b & z[s]) & 1) ? -p : p;
                    }
                } else {
                    const int lb = __ffs(G.X) - 1;
                    for (uint32_t i = threadIdx.x; i < E / 2; i += blockDim.x) {
                        const uint32_t e = ins0(i, lb), f = e ^ G.X;
                        const Cx<R> u = tile[e], v = tile[f];
                        const R wr = v.x * u.x + v.y * u.y;    // Re(conj(v) u)
                        const R wi = v.x * u.y - v.y * u.x;    // Im(conj(v) u)
                        const uint64_t b = rep ^ spanv[e >> a.kl] ^ (e & lowmask);
#pragma unroll
                        for (int s = 0; s < kEvcChunk; ++s) {
                            const R val = (ny[s] & 1) ? wi : wr;
                            const int neg = ((ny[s] == 1) | (ny[s] == 2)) ^ (__popcll(b & z[s]) & 1);
                            accr[s] += neg ? -2 * val : 2 * val;
                        }
                    }
                }
#pragma unroll
                for (int s = 0; s < kEvcChunk; ++s) {
                    if (s < ns) {
                        const R v = warp_sum<R>(accr[s]);
                        if (lane == 0) acc[(cs + s - a.s_begin) * nwarps + warp] += (double)v;
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += acc[s * nwarps + w];
        part[(size_t)blockIdx.x * part_stride + a.s_begin + s] = t;
    }
}

// ------------------------------------------------------------------ K-HPSI --
// lambda[b] += sum_t a_t i^nY (-1)^{|(b^x)&z|} psi[b^x] for every group of the
// pass (P|c> = i^nY (-1)^{|c&z|} |c^x>, c = b^x).  The first pass stores,
// later passes add; the last one also accumulates Re<psi|lambda>.
template <typename R, int EPT>
__global__ void __launch_bounds__(512) k_hpsi_pass(const Cx<R> *__restrict__ psi, Cx<R> *__restrict__ lam,
                                                   const CosetArgs a, const DevGroup *__restrict__ groups,
                                                   const DevString *__restrict__ strs, int first, int last,
                                                   double *__restrict__ epart) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t E = 1u << (a.kl + a.m);
    const uint32_t M = 1u << a.m;
    Cx<R> *tile = reinterpret_cast<Cx<R> *>(smem);
    uint64_t *spanv = reinterpret_cast<uint64_t *>(tile + E);
    __shared__ double wsum[32];
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        uint64_t v = 0;
        for (int i = 0; i < a.m; ++i)
            if (j >> i & 1u) v ^= a.basis[i];
        spanv[j] = v;
    }
    __syncthreads();
    const uint32_t lowmask = (1u << a.kl) - 1u;
    const uint64_t ncos = 1ull << a.nfree;
    double eacc = 0.0;
    for (uint64_t ci = blockIdx.x; ci < ncos; ci += gridDim.x) {
        const uint64_t rep = deposit(ci, a.freeb, a.nfree);
        for (uint32_t e = threadIdx.x; e < E; e += blockDim.x)
            tile[e] = psi[rep ^ spanv[e >> a.kl] ^ (e & lowmask)];
        __syncthreads();
        Cx<R> acc[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) acc[j] = mk<R>(0, 0);
        for (int gi = a.g_begin; gi < a.g_end; ++gi) {
            const DevGroup G = groups[gi];
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const uint32_t e = threadIdx.x + j * blockDim.x;
                if (e >= E) continue;
                const Cx<R> v = tile[e ^ G.X];
                const uint64_t bf = rep ^ spanv[e >> a.kl] ^ (e & lowmask) ^ G.x;
                R ar = 0, ai = 0;
                for (int s = G.s_begin; s < G.s_end; ++s) {
                    const DevString S = strs[s];
                    const R cf = (__popcll(bf & S.z) & 1) ? -(R)S.coef : (R)S.coef;
                    // i^nY * v
                    R rr, ri;
                    switch (S.nY) {
                    case 0: rr = v.x; ri = v.y; break;
                    case 1: rr = -v.y; ri = v.x; break;
                    case 2: rr = -v.x; ri = -v.y; break;
                    default: rr = v.y; ri = -v.x; break;
                    }
                    ar += cf * rr;
                    ai += cf * ri;
                }
                acc[j].x += ar;
                acc[j].y += ai;
            }
        }
        R eloc = 0;
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const uint32_t e = threadIdx.x + j * blockDim.x;
            if (e >= E) continue;
            const uint64_t gi = rep ^ spanv[e >> a.kl] ^ (e & lowmask);
            Cx<R> out = acc[j];
            if (!first) {
                const Cx<R> old = lam[gi];
                out.x += old.x;
                out.y += old.y;
            }
            lam[gi] = out;
            if (last) {
                const Cx<R> p = tile[e];
                eloc += p.x * out.x + p.y * out.y;
            }
        }
        eacc += (double)eloc;
        __syncthreads();
    }
    if (last) {
        double v = eacc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
            epart[blockIdx.x] = t;
        }
    }
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
    const size_t es = dt == SV_C64 ? 8 : 16;
    return (size_t)E * es + ((size_t)1 << m) * 8 + (size_t)nslots * nwarps * 8;
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
    // a fixed grid per call so every pass writes the same partial rows
    int per = (E >= 4096) ? 2 : 4;
    if (hpsi) per = 2;
    if (blocks_per_sm > 0) per = std::min(per, blocks_per_sm);
    (void)dt;
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
    const size_t sm = 2 * ((size_t)1 << a.ntb) * es + ((size_t)1 << (a.ntb - a.L)) * 8;
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

cudaError_t launch_evc_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, const CosetArgs &a,
                            const DevGroup *groups, const DevString *strs, double *part, int part_stride) {
    const int threads = 256;
    const int E = 1 << (a.kl + a.m);
    const size_t sm = coset_smem(dt, E, a.m, a.s_end - a.s_begin, threads / 32);
    if (dt == SV_C64) {
        allow_smem(k_evc_pass<float>, sm);
        k_evc_pass<float><<<grid, threads, sm, st>>>((const float2 *)psi, a, groups, strs, part, part_stride);
    } else {
        allow_smem(k_evc_pass<double>, sm);
        k_evc_pass<double><<<grid, threads, sm, st>>>((const double2 *)psi, a, groups, strs, part, part_stride);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t hpsi_dispatch(cudaStream_t st, int grid, const void *psi, void *lam, const CosetArgs &a,
                          const DevGroup *groups, const DevString *strs, int first, int last, double *epart) {
    const int E = 1 << (a.kl + a.m);
    const size_t es = sizeof(Cx<R>);
    const size_t sm = (size_t)E * es + ((size_t)1 << a.m) * 8;
    // at least one full warp (the energy reduction shuffles across 32 lanes)
    int threads = std::max(32, std::min(E, 256));
    int ept = std::max(1, E / threads);
#define SV_HPSI_CASE(N)                                                                                      \
    case N:                                                                                                  \
        allow_smem(k_hpsi_pass<R, N>, sm);                                                                   \
        k_hpsi_pass<R, N><<<grid, threads, sm, st>>>((const Cx<R> *)psi, (Cx<R> *)lam, a, groups, strs,     \
                                                     first, last, epart);                                    \
        break;
    switch (ept) {
        SV_HPSI_CASE(1)
        SV_HPSI_CASE(2)
        SV_HPSI_CASE(4)
        SV_HPSI_CASE(8)
        SV_HPSI_CASE(16)
        SV_HPSI_CASE(32)
    default:
        return cudaErrorInvalidValue;
    }
#undef SV_HPSI_CASE
    return cudaGetLastError();
}

cudaError_t launch_hpsi_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, void *lam,
                             const CosetArgs &a, const DevGroup *groups, const DevString *strs, int first,
                             int last, double *epart) {
    if (dt == SV_C64) return hpsi_dispatch<float>(st, grid, psi, lam, a, groups, strs, first, last, epart);
    return hpsi_dispatch<double>(st, grid, psi, lam, a, groups, strs, first, last, epart);
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

}  // namespace sv
