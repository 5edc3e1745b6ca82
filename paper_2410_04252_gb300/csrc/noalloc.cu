// sv_expect_noalloc: Pauli-string expectation values on a caller-owned state
// without allocating device memory.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// want expectation values -- for example code whose device memory is owned by
// another allocator (a framework's caching pool that has already reserved
// most of HBM, so a raw cudaMalloc fails or fragments it), and code that must
// not let an allocation stall the whole device (cudaMalloc and cudaFree may
// wait for work on every stream) in the middle of a pipeline; this call waits
// only for its own stream.  The ordinary entry points (sv_expect and friends)
// allocate their scratch and plan buffers lazily with cudaMalloc; this one
// does not.  It copies its tables from pageable host memory and synchronises
// its stream, so it cannot be called inside a stream capture.
//
// Scratch: one file-scope device array of kNoAllocScratchBytes bytes.  Every
// GPU that loads this library holds it until the process exits.  All calls
// share it and it keeps the contents of the last call; every word a call reads
// back from it was written earlier in the same call, so nothing has to start
// at zero.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "sv_internal.h"

namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)1 << 20;   // 1 MiB
constexpr int kNoAllocMaxTerms = 256;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

// In host code this name is only a host-side stand-in for the device array;
// host code must use the address from cudaGetSymbolAddress (scratch_address).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices];   // device address of the array, per device

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

sv_status noalloc_fail(sv_status s, const std::string &m) {
    sv::set_last_error(m);
    return s;
}

// Device address of the scratch array on the current device.  The first
// call on a device looks it up (cudaGetSymbolAddress, with that device
// current) and caches it.
sv_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(SV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return noalloc_fail(SV_EINVAL, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(SV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SV_OK;
}

}  // namespace

extern "C" sv_status sv_expect_noalloc(const void *state, int n, sv_dtype dt, const sv_pauli *paulis,
                                       const double *coeffs, size_t nterms, double *energy, double *per_term,
                                       void *stream) {
    if (!state || !paulis || !coeffs || !energy) return noalloc_fail(SV_EINVAL, "null argument");
    // the EVC kernels stage the state with 16-byte asynchronous copies: an
    // unaligned state (e.g. a view at an odd complex64 offset) is refused here,
    // before anything is launched
    if ((uintptr_t)state % 16) return noalloc_fail(SV_EINVAL, "state must be 16-byte aligned");
    if (n < 1 || n > sv::kMaxQubits) return noalloc_fail(SV_EINVAL, "n must be in [1, 40]");
    if (dt != SV_C64 && dt != SV_C128) return noalloc_fail(SV_EINVAL, "bad dtype");
    if (nterms < 1 || nterms > (size_t)kNoAllocMaxTerms)
        return noalloc_fail(SV_EINVAL, "sv_expect_noalloc takes 1 to 256 Pauli strings per call");
    const uint64_t lim = (1ull << n) - 1;
    for (size_t t = 0; t < nterms; ++t) {
        if ((paulis[t].x & ~lim) || (paulis[t].z & ~lim)) return noalloc_fail(SV_EINVAL, "Pauli mask beyond n qubits");
        if (!std::isfinite(coeffs[t])) return noalloc_fail(SV_EINVAL, "non-finite coefficient");
    }
    void *base = nullptr;
    sv_status s = scratch_address(&base);
    if (s != SV_OK) return s;

    // host planning: strings grouped by X/Y mask and packed into coset
    // passes over all n index bits, state taken in its index order
    sv_options o;
    sv_options_default(dt, &o);
    sv::PlanOptions po;
    po.evc_low_bits = o.evc_low_bits;
    po.evc_span = o.evc_span;
    std::vector<int32_t> l2p(n);
    for (int q = 0; q < n; ++q) l2p[q] = q;
    sv::EvcPlan P;
    std::string err = sv::plan_hpsi(n, paulis, coeffs, nterms, po, l2p, P);
    if (!err.empty()) return noalloc_fail(SV_EINVAL, "plan: " + err);
    const int nslots = (int)P.strings.size();
    const int ngroups = (int)P.groups.size();

    std::vector<sv::DevGroup> gs(ngroups);
    for (int i = 0; i < ngroups; ++i) {
        gs[i].x = P.groups[i].x;
        gs[i].X = P.groups[i].X;
        gs[i].s_begin = P.groups[i].s_begin;
        gs[i].s_end = P.groups[i].s_end;
        gs[i].parts = 0;
        for (int32_t q = P.groups[i].s_begin; q < P.groups[i].s_end; ++q) gs[i].parts |= 1 << (P.strings[q].nY & 1);
    }
    std::vector<sv::DevString> ss(nslots);
    for (int i = 0; i < nslots; ++i) {
        ss[i].z = P.strings[i].z;
        ss[i].coef = P.strings[i].coef;
        ss[i].nY = P.strings[i].nY;
        ss[i].bz = P.strings[i].bz;
    }

    // carve the array: tables, results, then per-CTA partial rows
    unsigned char *p = (unsigned char *)base;
    size_t off = 0;
    sv::DevGroup *d_groups = (sv::DevGroup *)(p + off); off = align256(off + ngroups * sizeof(sv::DevGroup));
    sv::DevString *d_strs = (sv::DevString *)(p + off); off = align256(off + nslots * sizeof(sv::DevString));
    int32_t *d_term_slot = (int32_t *)(p + off); off = align256(off + nterms * sizeof(int32_t));
    double *d_coeffs = (double *)(p + off); off = align256(off + nterms * sizeof(double));
    double *d_slotval = (double *)(p + off); off = align256(off + nslots * sizeof(double));
    double *d_per_term = (double *)(p + off); off = align256(off + nterms * sizeof(double));
    double *d_energy = (double *)(p + off); off = align256(off + sizeof(double));
    int *d_status = (int *)(p + off); off = align256(off + sizeof(int));
    double *d_part = (double *)(p + off);
    if (off >= kNoAllocScratchBytes) return noalloc_fail(SV_EINVAL, "scratch array too small for this call");
    int E = 1;
    for (auto &cp : P.passes) E = std::max(E, 1 << (cp.kl + cp.m));
    int grid = sv::coset_grid(dt, E, 0, false);
    const size_t rows = (kNoAllocScratchBytes - off) / ((size_t)nslots * sizeof(double));
    if (rows < 1) return noalloc_fail(SV_EINVAL, "scratch array too small for this call");
    if ((size_t)grid > rows) grid = (int)rows;

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
#define NOALLOC_CK(call)                                                                                  \
    do {                                                                                                  \
        e = (call);                                                                                       \
        if (e != cudaSuccess) return noalloc_fail(SV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e)); \
    } while (0)
    NOALLOC_CK(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    NOALLOC_CK(cudaMemcpyAsync(d_groups, gs.data(), ngroups * sizeof(sv::DevGroup), cudaMemcpyHostToDevice, st));
    NOALLOC_CK(cudaMemcpyAsync(d_strs, ss.data(), nslots * sizeof(sv::DevString), cudaMemcpyHostToDevice, st));
    NOALLOC_CK(cudaMemcpyAsync(d_term_slot, P.term_slot.data(), nterms * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NOALLOC_CK(cudaMemcpyAsync(d_coeffs, coeffs, nterms * sizeof(double), cudaMemcpyHostToDevice, st));
    for (auto &cp : P.passes) {
        sv::CosetArgs a;
        memset(&a, 0, sizeof(a));
        a.n = n;
        a.kl = cp.kl;
        a.m = cp.m;
        uint64_t piv = 0;
        for (int j = 0; j < cp.m; ++j) {
            a.basis[j] = cp.basis[j];
            piv |= 1ull << cp.pivot[j];
        }
        for (int b = cp.kl; b < n; ++b)
            if (!(piv >> b & 1)) a.freeb[a.nfree++] = (int8_t)b;
        a.g_begin = cp.g_begin;
        a.g_end = cp.g_end;
        a.s_begin = cp.s_begin;
        a.s_end = cp.s_end;
        NOALLOC_CK(sv::launch_evc_pass(dt, st, grid, state, a, d_groups, d_strs, d_part, nslots, d_status,
                                       (long long)o.wait_limit));
    }
    NOALLOC_CK(sv::launch_reduce_rows(st, d_part, grid, nslots, 0, nslots, d_slotval));
    NOALLOC_CK(sv::launch_energy(st, d_slotval, d_term_slot, d_coeffs, (int)nterms, d_per_term, d_energy));
    NOALLOC_CK(cudaMemcpyAsync(energy, d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (per_term)
        NOALLOC_CK(cudaMemcpyAsync(per_term, d_per_term, nterms * sizeof(double), cudaMemcpyDeviceToHost, st));
    int status = 0;
    NOALLOC_CK(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NOALLOC_CK(cudaStreamSynchronize(st));
#undef NOALLOC_CK
    if (status) return noalloc_fail(SV_ETIMEOUT, "a device wait for a bulk copy expired");
    return SV_OK;
}
