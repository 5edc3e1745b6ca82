// Launchers of the device kernels (kernels.cu).  All take a stream and return
// the CUDA error of the launch.
#pragma once

#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

// Gate / adjoint pass: 2^k staged amplitudes; tile bits 0..nlow-1 are
// physical bits 0..nlow-1, tile bits nlow..k-1 are hi[]; out[] lists the
// physical bits that are not staged (they index the tiles).
struct GatePassArgs {
    int n, k, nlow, nhi, nout, op_begin, op_end;
    int ph_begin, ph_end;    // register phases (register-blocked pass), else -1
    int db_begin, db_end;    // diagonal blocks of the pass
    int st_begin, st_end;    // steps of the pass's register phases
    int area;                // bytes of the diagonal-block data
    int mem_begin, mem_end;  // diagonal-block members of the pass
    int8_t hi[40];
    int8_t out[64];
};

// Coset pass (EVC / H|psi>): 2^(kl+m) staged amplitudes, runs of 2^kl
// contiguous ones at rep ^ span(a); free[] lists the bits >= kl that are not
// pivots (they index the coset representatives).
struct CosetArgs {
    int n, kl, m, nfree, g_begin, g_end, s_begin, s_end;
    int few;                 // 1: every group has one string and there are at most 8 groups
    uint64_t basis[kMaxSpan];
    int8_t freeb[64];
};

struct DevGroup {
    uint64_t x;
    uint32_t X;
    int32_t s_begin, s_end;
    int32_t parts;    // bit 0: a string with nY even (uses Re), bit 1: one with nY odd (uses Im)
};
struct DevString {
    uint64_t z;
    double coef;
    int32_t nY;
    uint32_t bz;      // parities of the pass's span basis against z
};

// Few-string expectation passes (every group one string): at most this many groups.
constexpr int kEvcFew = 8;

// Batched kernel arguments (see K-BATCH in kernels.cu).
struct BatchArgs {
    int n, nstates, nhpass;
    int kmax;                        // staged amplitudes per buffer: 2^kmax (gate passes and H|psi> cosets)
    int hio;                         // entries of the high-offset table: 2^hio
    uint64_t init_index;
    const GatePassArgs *passes;      // all plans' gate passes
    const Phase *phases;             // all plans' register phases (ph_begin/ph_end of a pass index them)
    const int32_t *plan_pass_off;    // [nplans + 1]
    const DevOp *ops;                // all plans' pass operations (gate = index within the state's circuit)
    const int32_t *plan_op_off;      // [nplans + 1]: first op of each plan (ops are plan-contiguous)
    const int32_t *state_plan;       // [nstates]
    const int32_t *order;            // [nstates] processing order
    const int32_t *gate_off;         // [nstates + 1] into gparam
    const int32_t *gparam;           // parameter index (within the state's params) per gate, -1 = none
    const int32_t *param_off;        // [nstates + 1] into params / grads
    const double *params;
    const CosetArgs *hpass;          // shared Hamiltonian passes
    const DevGroup *groups;
    const DevString *strs;
    void *work;                      // per CTA: psi, lambda (2^n each)
    double *energies;                // [nstates]
    double *grads;                   // like params
    unsigned long long *t_start, *t_end;
    int *counter;
};

int device_sms();
int gate_pass_grid(sv_dtype dt, int k, int nlow, int nops, int threads, int blocks_per_sm);
int adj_pass_grid(sv_dtype dt, int k, int nlow, int nops, int threads, int blocks_per_sm);
int coset_grid(sv_dtype dt, int E, int blocks_per_sm, bool hpsi);

cudaError_t launch_prep(sv_dtype dt, cudaStream_t st, const int32_t *gparam, const double *params,
                        int m, void *coef);
cudaError_t launch_set_basis(sv_dtype dt, cudaStream_t st, void *psi, size_t bytes, uint64_t index);
cudaError_t launch_gate_pass(sv_dtype dt, cudaStream_t st, int grid, int threads, void *psi,
                             const GatePassArgs &a, const DevOp *ops, const void *coef, const void *mats);
cudaError_t launch_adj_pass(sv_dtype dt, cudaStream_t st, int grid, int threads, void *psi, void *lam,
                            const GatePassArgs &a, const DevOp *ops, const void *coef, const void *mats,
                            double *part, int part_stride);
// Register-blocked passes (512 threads; a.ph_begin >= 0, 11 <= k <= 13): the
// phases' steps (RegStep) are executed in order (forward) or in reverse
// (adjoint); part receives the FP64 gradient partials of every operation.
cudaError_t launch_gate_reg(sv_dtype dt, cudaStream_t st, int grid, void *psi, const GatePassArgs &a,
                            const DevOp *ops, const Phase *phases, const RegStep *steps, const void *coef,
                            const void *mats, const DiagBlock *dblocks, const DiagMember *dmem);
cudaError_t launch_adj_reg(sv_dtype dt, cudaStream_t st, int grid, void *psi, void *lam, const GatePassArgs &a,
                           const DevOp *ops, const Phase *phases, const RegStep *steps, const void *coef,
                           const void *mats, double *part, int part_stride, const DiagBlock *dblocks,
                           const DiagMember *dmem);
// Shared memory of a register-blocked pass (forward / adjoint).
size_t gate_reg_smem(sv_dtype dt, const GatePassArgs &a);
size_t adj_reg_smem(sv_dtype dt, const GatePassArgs &a);
// In-place swap of disjoint physical bit pairs (pairs[2i], pairs[2i+1]).
cudaError_t launch_bitswap(sv_dtype dt, cudaStream_t st, void *psi, int n, const int32_t *pairs,
                           int npairs, int blocks_per_sm);
// Coset passes.  Their copies complete by cp.async groups, so no pass spins;
// status and limit are kept for the bounded-wait contract of the C ABI and
// are not read by the current kernels.
cudaError_t launch_evc_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, const CosetArgs &a,
                            const DevGroup *groups, const DevString *strs, double *part, int part_stride,
                            int *status, long long limit);
cudaError_t launch_hpsi_pass(sv_dtype dt, cudaStream_t st, int grid, const void *psi, void *lam,
                             const CosetArgs &a, const DevGroup *groups, const DevString *strs,
                             int first, int last, double *epart, int *status, long long limit);
// out[s] = sum over b < nblocks of part[b * stride + s], s in [s_begin, s_end); fixed order.
cudaError_t launch_reduce_rows(cudaStream_t st, const double *part, int nblocks, int stride,
                               int s_begin, int s_end, double *out);
// grad[param[i]] accumulation in a fixed order: grad[p] = sum_{i in list(p)} opval[i].
cudaError_t launch_scatter(cudaStream_t st, const double *opval, const int32_t *csr_off,
                           const int32_t *csr_idx, int np, double *grad);
// energy = sum_t coef_t * slotval[slot_t] and per-term values.
cudaError_t launch_energy(cudaStream_t st, const double *slotval, const int32_t *term_slot,
                          const double *coeffs, int nterms, double *per_term, double *energy);
cudaError_t launch_copy(sv_dtype dt, cudaStream_t st, void *dst, const void *src, size_t n_elems);
// One persistent launch over all states (512 threads per CTA).
cudaError_t launch_batch(sv_dtype dt, cudaStream_t st, int grid, int threads, const BatchArgs &a);
// One greedy step of Alg. 6 over the global sets of ranks [0, ncand): best receives
// max over (count << 32) | (0xFFFFFFFF - rank); binom is C(a, b) as [(n + 1)][(k + 1)].
cudaError_t launch_alg6_step(cudaStream_t st, const uint64_t *xs, const int32_t *w, int nx, int n, int k,
                             const int64_t *binom, uint64_t ncand, unsigned long long *best);
size_t batch_smem(sv_dtype dt, int kmax, int hio, int threads);
// 0 when (dt, kmax, threads) has no instantiated kernel
int batch_supported(sv_dtype dt, int kmax, int threads);
int batch_occupancy(sv_dtype dt, int kmax, int hio, int threads);
int batch_max_ops();
int batch_max_gates();

}  // namespace sv
