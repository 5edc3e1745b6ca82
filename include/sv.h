/*
 * libsv -- lazy qubit reordering state-vector simulation on one GB300 GPU.
 *
 * C ABI of the library.  Plain pointers and sizes only; every entry point
 * returns an sv_status and never throws.  On failure sv_last_error() gives a
 * thread-local message.  A handle is used by one host thread at a time.
 *
 * Model (arXiv 2410.04252, Sec. III-B):
 *   The state |psi> of n qubits is 2^n complex amplitudes held in ONE device
 *   buffer, interleaved (re, im) -- complex64 (float2) or complex128
 *   (double2), the memory layout of torch.complex64 / torch.complex128.
 *   Logical qubit q sits at physical index bit l2p[q]; the top g physical bits
 *   are "global" and split the buffer into 2^g virtual chunks (Eq. sub_sv),
 *   the low n_L = n - g bits are "local".  Gates and Pauli strings only ever
 *   touch local physical bits (narrow access, Sec. III-B-3); a qubit
 *   reordering (QR, Sec. III-B-4) swaps local and global bit pairs in place.
 *
 * Conventions for gates (the paper does not define GateFabric's gates):
 *   U = exp(-i theta G / 2) with G = Y (RY), Z (RZ), Y on span{|10>,|01>} of
 *   (q0,q1) (GIVENS), Y on span{|q0=q1=1,q2=q3=0>, |q2=q3=1,q0=q1=0>} (DEXC);
 *   CZ = diag(1,1,1,-1); MATk: caller matrix, row-major complex, target t
 *   <-> bit t of the matrix index.
 */
#ifndef LIBSV_SV_H
#define LIBSV_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SV_OK = 0,
    SV_EINVAL = 1,    /* invalid argument (sizes, qubit indices, NaN, ...) */
    SV_ENOMEM = 2,    /* device or host allocation failed */
    SV_ECUDA = 3,     /* a CUDA runtime call or launch failed */
    SV_EPLAN = 4,     /* internal plan validation failed */
    SV_ETIMEOUT = 5,  /* a bounded device wait expired */
    SV_EDEVICE = 6,   /* a kernel reported an error through its status word */
    SV_ESTATE = 7     /* call not valid in the handle's current state */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Schedules: EAGER = the ad hoc rule (depth order; before each wide operation
 * a QR for that operation alone, Sec. V-B-1); LAZY = time-space tiling
 * (Alg. 1-3 for QSU, Alg. 6 with diagonalization for EVC).  DIRECT is not
 * the paper's method: it drops the virtual-chunk constraint (every qubit is
 * local, as it may be when the whole state sits in one GPU's memory), so a
 * plan has one tile and no QR -- gate passes and coset passes may pair
 * amplitudes of different chunks.  It is the single-GPU optimum the two
 * schedules are compared against. */
typedef enum {
    SV_SCHED_EAGER = 0, SV_SCHED_LAZY = 1, SV_SCHED_DIRECT = 2, SV_SCHED_HIER = 3, SV_SCHED_LAZY_DIAG = 4
} sv_schedule;
/* SV_SCHED_LAZY_DIAG: LAZY with diagonal gates (RZ, CZ) exempt from
 * locality, as the paper's diagonalization exempts Z letters in EVC: a
 * diagonal gate on global qubits is a phase per chunk (per staged tile), so
 * it never asks for a QR; tiles grow past it and Alg. 3 ignores it.  Not the
 * paper's QSU method: compared against it.  EVC under it is the LAZY one. */
/* SV_SCHED_HIER: QSU by hierarchical tiling (Alg. 4 with Alg. 5) for a
 * two-layered interconnect whose intra-node part holds options.intra_bits of
 * the g global qubits (Q_intra starts at physical positions n-g ..
 * n-g+intra_bits-1); the remapping prefers an intra QR (next local set drawn
 * from Q_L u Q_intra) over an inter QR.  On one GPU every QR is the same
 * in-place permutation; the plan export tells intra from inter QRs
 * (sv_plan_tile_intra).  EVC under SV_SCHED_HIER is the LAZY one (Alg. 6). */

enum { SV_RY = 0, SV_RZ = 1, SV_CZ = 2, SV_GIVENS = 3, SV_DEXC = 4,
       SV_MAT1 = 5, SV_MAT2 = 6, SV_MAT4 = 7 };

/* One operator of the QCT form (Sec. III): kind, target qubits q[0..nq-1]
 * (unused entries -1), parameter index into params[] (-1: none) and, for
 * MATk, the offset in complex elements of its matrix inside mats[]. */
typedef struct {
    int32_t kind;
    int32_t q[4];
    int32_t param;
    int32_t mat;
} sv_gate;

/* A Pauli string P = i^{|x&z|} X^x Z^z on logical qubits (Eq. pauli_form):
 * bit q of x is set where P has X or Y, bit q of z where it has Z or Y. */
typedef struct {
    uint64_t x;
    uint64_t z;
} sv_pauli;

/* Tunables; zero fields take defaults.  sv_options_default() fills them. */
typedef struct {
    int32_t tile_bits;          /* k: a gate pass stages 2^k amplitudes (default 13 c64, 12 c128) */
    int32_t low_bits;           /* contiguous low bits kept in every gate pass (default 4) */
    int32_t evc_low_bits;       /* shortest contiguous run (bits) of an EVC / H|psi> coset pass (default 5 c64,
                                   4 c128); a pass stages 2^(evc_low_bits + evc_span) amplitudes and lengthens
                                   its runs when it needs a smaller span */
    int32_t evc_span;           /* max coset dimension m of an EVC / H|psi> pass (default 8, at most 10) */
    int32_t pad_highest;        /* Alg. 3 padding: 1 highest free qubit (default), 0 lowest (printed text) */
    int32_t checkpoint_every;   /* c > 0: the forward sweep keeps a copy of psi after every c-th gate pass
                                   (device memory, else pinned host memory) and the adjoint sweep
                                   re-anchors psi from it instead of the uncomputed value; 0 = none */
    int32_t threads;            /* CTA size of adjoint passes (default 512; gate passes use min(256, threads)) */
    int32_t blocks_per_sm;      /* persistent grid multiplier (0 = occupancy) */
    int64_t wait_limit;         /* spin iterations before a device wait gives up (batched kernel) */
    int32_t profile;            /* 1: time every launch with CUDA events on the stream (sv_stats.ms);
                                   calls then synchronise before returning */
    int32_t fuse_max;           /* fusion depth: at most this many gate operations per gate pass
                                   (0 = as many as fit, up to 256) */
    int32_t intra_bits;         /* SV_SCHED_HIER: intra-node global qubits n_intra, 0 <= n_intra <= g */
    int32_t plan_device;        /* where Alg. 6 searches the global sets of the lazy EVC plan: 0 = on the
                                   GPU when C(n, g) >= 2^19 and a CUDA device is present (default), 1 = on
                                   the GPU, 2 = on the host; both give the same plan */
} sv_options;

/* Kernel kinds counted in sv_stats. */
enum { SV_K_GATE = 0,   /* fused gate pass */
       SV_K_QR = 1,     /* qubit reordering (bit-pair swap) */
       SV_K_EVC = 2,    /* Pauli-string expectation pass */
       SV_K_HPSI = 3,   /* lambda = H psi pass */
       SV_K_ADJ = 4,    /* adjoint reverse pass */
       SV_K_PERM = 5,   /* layout restore (bit-pair swaps) */
       SV_K_AUX = 6,    /* coefficient prep, reductions, basis reset */
       SV_K_BATCH = 7,  /* persistent batched kernel */
       SV_K_COUNT = 8 };

/* Counters of one call (optional output). */
typedef struct {
    int32_t qsu_tiles, qsu_qrs, qsu_passes;
    int32_t evc_tiles, evc_qrs, evc_passes;
    int32_t hpsi_passes, adj_passes;
    int32_t launches;              /* kernels launched by this call */
    int32_t plan_cache_hit;        /* every plan came from the cache */
    double plan_ms;                /* host planning time (0 on a cache hit) */
    int32_t kernels[SV_K_COUNT];   /* launches per kind */
    double bytes[SV_K_COUNT];      /* algorithmic bytes per kind: 2S per gate pass,
                                      2(1-2^-s)S per QR of s pairs, S per EVC pass,
                                      2S / 3S per first / later lambda pass, 4S per
                                      adjoint pass (S = 2^n * amplitude size) */
    double ms[SV_K_COUNT];         /* device time per kind (options.profile = 1) */
} sv_stats;

typedef struct sv_handle sv_handle;

void sv_options_default(sv_dtype dt, sv_options *out);

/* Create a simulator for n qubits (1 <= n <= 40) with 2^g virtual chunks
 * (0 <= g <= n - 4 so that a 4-qubit operator fits the local qubits).
 * Selects the current CUDA device; allocates nothing on the device until a
 * buffer is needed.  *out is owned by the caller and freed by sv_destroy. */
sv_status sv_create(int n, int g, sv_dtype dt, sv_handle **out);
void sv_destroy(sv_handle *h);

/* Attach a caller-owned device buffer of 2^n amplitudes as the state (e.g. a
 * torch tensor's data_ptr).  The library never frees it.  bytes must be
 * >= 2^n * sizeof(amplitude); the pointer must be 256-byte aligned. */
sv_status sv_attach_state(sv_handle *h, void *dev_ptr, size_t bytes);
/* The same call under the name of the original interface sketch. */
sv_status sv_attach_buffer(sv_handle *h, void *dev_ptr, size_t bytes);
/* Attach a caller-owned device buffer for the adjoint vector lambda = H psi
 * (same size and alignment rules).  Without it sv_grad allocates one. */
sv_status sv_attach_lambda(sv_handle *h, void *dev_ptr, size_t bytes);

/* All work is enqueued on this stream (cudaStream_t passed as void*; NULL =
 * the legacy default stream). */
sv_status sv_set_stream(sv_handle *h, void *stream);
sv_status sv_set_options(sv_handle *h, const sv_options *opt);
sv_status sv_get_options(const sv_handle *h, sv_options *opt);

/* |psi> = |logical_index>, identity layout (l2p[q] = q). Asynchronous. */
sv_status sv_reset_basis(sv_handle *h, uint64_t logical_index);
/* Copy 2^n amplitudes in LOGICAL order from src (host or device) into the
 * state and reset the layout to identity.  Synchronous for host src. */
sv_status sv_set_state(sv_handle *h, const void *src, int src_is_device);
/* Copy the state to dst (host or device, 2^n amplitudes).  logical_order=1
 * undoes the current layout (index bit q = logical qubit q); 0 copies the
 * physical buffer as is.  Synchronises the stream. */
sv_status sv_get_state(sv_handle *h, void *dst, int dst_is_device, int logical_order);
/* l2p[q] = physical bit of logical qubit q (n entries). */
sv_status sv_get_permutation(const sv_handle *h, int32_t *l2p);

/*
 * QSU (Eq. vqe_qsu): |psi> <- U_{m-1} ... U_0 |psi> under the given schedule,
 * starting from the current layout.  LAZY runs the flat time-space tiling of
 * Alg. 1 (tiles from Alg. 2, remapping by Alg. 3), EAGER the ad hoc rule;
 * both then group each tile's gates into shared-memory passes of 2^k
 * amplitudes.  params[np] (host, radians), mats (host, complex interleaved,
 * nmats complex elements, may be NULL).  The plan is cached on the handle
 * (Sec. V-C: computed once, reused every VQE iteration).  Asynchronous.
 * Errors: EINVAL for a qubit >= n, duplicate targets, a parameter index
 * >= np, a matrix out of range, a NaN parameter.
 */
sv_status sv_apply_circuit(sv_handle *h, const sv_gate *gates, size_t m,
                           const double *params, size_t np,
                           const double *mats, size_t nmats,
                           sv_schedule sched, sv_stats *stats);

/* Flags for sv_expect / sv_grad. */
#define SV_KEEP_LAYOUT 1u    /* sv_expect: restore the entry layout afterwards */
#define SV_FORWARD_DONE 2u   /* sv_grad: the state already is U|psi0> from the
                                last sv_apply_circuit of the same circuit, in
                                that call's final layout */

/*
 * EVC (Eqs. evc, parallel_evc, par_exp): energy = sum_t coeffs[t] <psi|P_t|psi>.
 * LAZY: Alg. 6 tiling over X/Y supports (diagonalization: Z on global qubits
 * becomes a per-chunk sign), QR between tiles; EAGER: strings in index order
 * with ad hoc QRs.  Inside a tile, strings sharing an X/Y mask share one read
 * and masks are packed into coset passes.  per_term (nullable) receives
 * nterms real values <P_t>.  Partial sums are accumulated in FP64 and reduced
 * in a fixed order.  A string with more than n - g X/Y positions fits no
 * virtual-chunk layout (the paper does not treat this case): such strings are
 * evaluated in one last tile without a QR, pairing amplitudes across chunks.
 * Synchronises.  Errors: EINVAL for masks >= 2^n or non-finite coefficients.
 */
sv_status sv_expect(sv_handle *h, const sv_pauli *paulis, const double *coeffs,
                    size_t nterms, sv_schedule sched, uint32_t flags,
                    double *energy, double *per_term, sv_stats *stats);

/*
 * lambda = H|psi> into the handle's lambda buffer (physical layout of psi)
 * and energy = Re<psi|lambda>.  Used by sv_grad; exposed for testing.
 * dst (nullable, device) additionally receives a copy of lambda.  Synchronises.
 */
sv_status sv_apply_hamiltonian(sv_handle *h, const sv_pauli *paulis, const double *coeffs,
                               size_t nterms, void *dst_device, double *energy,
                               sv_stats *stats);

/*
 * Adjoint gradient of E(theta) = <psi0|U^dagger H U|psi0> (Eqs. vqe,
 * vqe_qsu, vqe_evc): forward QSU (skipped with SV_FORWARD_DONE), lambda =
 * H|psi>, then a reverse sweep over the same plan: per gate k in reverse,
 * grad[param_k] += Im<lambda|G_k|psi> then psi <- U_k^dagger psi and
 * lambda <- U_k^dagger lambda, with the inverse QRs between tiles.  On
 * return the state is back at |psi0> (up to rounding) in its entry layout.
 * grad (host) has np entries.  Synchronises.
 */
sv_status sv_grad(sv_handle *h, const sv_gate *gates, size_t m,
                  const double *params, size_t np, const double *mats, size_t nmats,
                  const sv_pauli *paulis, const double *coeffs, size_t nterms,
                  sv_schedule sched, uint32_t flags,
                  double *energy, double *grad, sv_stats *stats);

/*
 * One VQE iteration: |psi> = |init>, QSU, EVC (per_term nullable), then the
 * adjoint gradient of the same energy.  energy comes from the EVC; grad has
 * np entries.  Synchronises.
 */
sv_status sv_vqe_step(sv_handle *h, uint64_t init_index,
                      const sv_gate *gates, size_t m, const double *params, size_t np,
                      const double *mats, size_t nmats,
                      const sv_pauli *paulis, const double *coeffs, size_t nterms,
                      sv_schedule sched, double *energy, double *per_term, double *grad,
                      sv_stats *stats);

/*
 * Host-only planning (no GPU needed), for inspection and bit-exact checks.
 * sv_plan_qsu: the tile schedule of Alg. 1 (LAZY) or the ad hoc rule (EAGER).
 * sv_plan_evc: Alg. 6 with diagonalization (LAZY) or index order (EAGER).
 * l2p_init (nullable) is the starting layout (identity if NULL).
 */
typedef struct sv_plan sv_plan;
sv_status sv_plan_qsu(int n, int g, const sv_gate *gates, size_t m, sv_schedule sched,
                      const sv_options *opt, const int32_t *l2p_init, sv_plan **out);
sv_status sv_plan_evc(int n, int g, const sv_pauli *paulis, size_t nterms, sv_schedule sched,
                      const sv_options *opt, const int32_t *l2p_init, sv_plan **out);
/* ntiles, total operations scheduled, device passes. */
sv_status sv_plan_info(const sv_plan *p, int32_t *ntiles, int32_t *nops, int32_t *npasses);
/* Schedule g: operation indices in execution order at tile granularity (nops). */
sv_status sv_plan_order(const sv_plan *p, int32_t *order);
/* Tile t: [begin, end) into the order, local set as a logical bit mask, the
 * QR performed before it (npairs pairs (local phys, global phys) into
 * pairs[2*i], pairs[2*i+1], room for 64 pairs) and the layout in force during
 * it (l2p[n]). */
sv_status sv_plan_tile(const sv_plan *p, int32_t t, int32_t *begin, int32_t *end,
                       uint64_t *local_mask, int32_t *npairs, int32_t *pairs, int32_t *l2p);
/* Pass i of a QSU plan: tile index, staged physical bit mask, and the
 * operation indices it applies, in order (ops may be NULL to query nops). */
sv_status sv_plan_pass(const sv_plan *p, int32_t i, int32_t *tile, uint64_t *bits,
                       int32_t *nops, int32_t *ops);
/* Hierarchical plans: the logical intra set Q_intra in force during tile t
 * (0 for other schedules).  A QR before tile t is an inter QR when the inter
 * set Q \ (Q_L u Q_intra) differs from the previous tile's (Fig. 7). */
sv_status sv_plan_tile_intra(const sv_plan *p, int32_t t, uint64_t *intra_mask);
void sv_plan_free(sv_plan *p);

/*
 * Batched VQE (many small independent states, one persistent launch; the
 * paper has no counterpart -- it is the batching extension): state b runs
 * circuit gates[gate_off[b] .. gate_off[b+1]) with parameters
 * params[param_off[b] .. param_off[b+1]) from |init_index>, then
 * lambda = H|psi> for the shared Hamiltonian with energy Re<psi|lambda>, then
 * the adjoint gradient -- all inside ONE kernel launch (captured in a CUDA
 * graph with the reset of its work counter) in which each CTA takes whole
 * states from an atomic counter, longest circuits first; no CTA waits for
 * another.  energies[batch] and grads (laid out like params) are written to
 * host memory; times_ns (nullable, 2*batch entries) receives each state's
 * device start and end time in ns relative to the earliest start.  n in
 * [4, 20], no virtual chunks, at most 512 gates per state.  Allocates its
 * device buffers for the call and frees them before returning.  Synchronises.
 */
sv_status sv_batch_run(int n, sv_dtype dt, int batch,
                       const sv_gate *gates, const int32_t *gate_off,
                       const double *params, const int32_t *param_off,
                       const sv_pauli *paulis, const double *coeffs, size_t nterms,
                       uint64_t init_index, const sv_options *opt, void *stream,
                       double *energies, double *grads, double *times_ns, sv_stats *stats);

/*
 * Expectation values without device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc where they need expectation values (their device memory is
 * owned by another allocator, or they cannot let an allocation stall every
 * stream of the device at that point: this call waits for its own stream
 * only).  It computes per_term[t] = <psi|P_t|psi> (host, nullable) and
 * energy = sum_t coeffs[t] per_term[t] (host) for the 2^n amplitudes at
 * state (device, complex64/complex128, 16-byte aligned, else EINVAL before
 * any launch; taken in index order: bit q of the index is qubit q), using
 * the library's EVC kernels with all scratch in one fixed 1 MiB static
 * device array held by every GPU that loads the library.  At most 256
 * strings per call; more is EINVAL.  No cudaMalloc/cudaFree is called.  The
 * call runs on the current device, and its first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current.  All calls share the array; calls whose work overlaps on the GPU
 * race on it.  The call copies its tables from pageable host memory and
 * synchronises the given stream (cudaStream_t as void*, NULL = legacy
 * default stream), so it cannot be made inside a stream capture.
 */
sv_status sv_expect_noalloc(const void *state, int n, sv_dtype dt, const sv_pauli *paulis,
                            const double *coeffs, size_t nterms, double *energy, double *per_term,
                            void *stream);

/*
 * Autotuner (the paper fixes neither the pass size nor the fusion depth: both
 * are parameters of this implementation).  Picks tile_bits (k), fuse_max
 * (fusion depth) and, when nterms > 0, the coset pass shape (evc_low_bits,
 * evc_span) for this handle by timing one step per candidate, coordinate by
 * coordinate from the handle's current options.  The step is sv_vqe_step
 * when nterms > 0, else sv_reset_basis + sv_apply_circuit.  Each candidate
 * runs once untimed (planning) and reps >= 1 times timed (host wall clock
 * around synchronised calls; the minimum counts).  The fastest options are
 * left set on the handle and copied to *best (nullable); *best_ms (nullable)
 * receives their time.  Overwrites the state.  Synchronises.
 */
sv_status sv_autotune(sv_handle *h, uint64_t init_index, const sv_gate *gates, size_t m,
                      const double *params, size_t np, const double *mats, size_t nmats,
                      const sv_pauli *paulis, const double *coeffs, size_t nterms,
                      sv_schedule sched, int reps, sv_options *best, double *best_ms);
/*
 * Autotuner of sv_batch_run (same arguments): over the (tile_bits, threads)
 * pairs the batched kernel is built for (2^tile_bits / threads in {4, 8, 16},
 * threads 256 or 512), then fuse_max.  Time = device time of the batched
 * launch (sv_stats.ms[SV_K_BATCH]), minimum over reps after one untimed run.
 * start (nullable) gives the other options.  Returns the fastest options in
 * *best and their time in *best_ms (both nullable).  Synchronises.
 */
sv_status sv_batch_autotune(int n, sv_dtype dt, int batch,
                            const sv_gate *gates, const int32_t *gate_off,
                            const double *params, const int32_t *param_off,
                            const sv_pauli *paulis, const double *coeffs, size_t nterms,
                            uint64_t init_index, const sv_options *start, void *stream, int reps,
                            sv_options *best, double *best_ms);

/* Wait until all work enqueued by the handle has finished. */
sv_status sv_synchronize(sv_handle *h);

const char *sv_last_error(void);
const char *sv_version(void);

#ifdef __cplusplus
}
#endif
#endif
