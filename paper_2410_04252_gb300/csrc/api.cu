// C ABI of libsv: handles, plan caches and the orchestration of the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "kernels.h"
#include "sv_internal.h"

using namespace sv;

namespace {

thread_local std::string g_err;

sv_status fail(sv_status s, const std::string &m) {
    g_err = m;
    return s;
}

#define SV_CK(call)                                                                                   \
    do {                                                                                              \
        cudaError_t _e = (call);                                                                      \
        if (_e != cudaSuccess) return fail(SV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define SV_TRY(call)                      \
    do {                                  \
        sv_status _s = (call);            \
        if (_s != SV_OK) return _s;       \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e == cudaSuccess) cap = bytes;
        else p = nullptr;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T> T *as() const { return (T *)p; }
};

template <class T>
cudaError_t upload(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    cudaError_t e = b.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

PlanOptions plan_options(const sv_options &o) {
    PlanOptions p;
    p.tile_bits = o.tile_bits;
    p.low_bits = o.low_bits;
    p.evc_low_bits = o.evc_low_bits;
    p.evc_span = o.evc_span;
    p.pad_highest = o.pad_highest != 0;
    p.fuse_max = o.fuse_max;
    return p;
}

GatePassArgs gate_args(int n, const GatePass &gp) {
    GatePassArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.k = gp.k;
    a.nlow = gp.nlow;
    a.nhi = 0;
    for (int b = gp.nlow; b < 64; ++b)
        if (gp.bits >> b & 1) a.hi[a.nhi++] = (int8_t)b;
    a.nout = 0;
    for (int b = 0; b < n; ++b)
        if (!(gp.bits >> b & 1)) a.out[a.nout++] = (int8_t)b;
    a.op_begin = gp.op_begin;
    a.op_end = gp.op_end;
    a.ph_begin = gp.ph_begin;
    a.ph_end = gp.ph_end;
    a.db_begin = gp.db_begin;
    a.db_end = gp.db_end;
    a.st_begin = gp.st_begin;
    a.st_end = gp.st_end;
    a.area = gp.area;
    a.mem_begin = gp.mem_begin;
    a.mem_end = gp.mem_end;
    return a;
}

CosetArgs coset_args(int n, const CosetPass &cp) {
    CosetArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.kl = cp.kl;
    a.m = cp.m;
    uint64_t piv = 0;
    for (int j = 0; j < cp.m; ++j) {
        a.basis[j] = cp.basis[j];
        piv |= 1ull << cp.pivot[j];
    }
    a.nfree = 0;
    for (int b = cp.kl; b < n; ++b)
        if (!(piv >> b & 1)) a.freeb[a.nfree++] = (int8_t)b;
    a.g_begin = cp.g_begin;
    a.g_end = cp.g_end;
    a.s_begin = cp.s_begin;
    a.s_end = cp.s_end;
    a.few = (cp.g_end - cp.g_begin) <= kEvcFew && (cp.s_end - cp.s_begin) == (cp.g_end - cp.g_begin);
    return a;
}

struct QsuEntry {
    uint64_t key = 0;
    QsuPlan plan;
    std::vector<GatePassArgs> args;
    DevBuf ops, gparam, csr_off, csr_idx, phases, steps, dblocks, dmembers;
    int m = 0, np = 0;
    double plan_ms = 0;
    uint64_t last_use = 0;
    void release() {
        ops.release(); gparam.release(); csr_off.release(); csr_idx.release(); phases.release(); steps.release();
        dblocks.release(); dmembers.release();
    }
};

struct EvcEntry {
    uint64_t key = 0;
    EvcPlan plan;
    std::vector<CosetArgs> args;
    DevBuf groups, strings, term_slot, coeffs;
    int nterms = 0;
    double plan_ms = 0;
    uint64_t last_use = 0;
    void release() { groups.release(); strings.release(); term_slot.release(); coeffs.release(); }
};

constexpr size_t kCacheSize = 6;

}  // namespace

struct sv_handle {
    int n = 0, g = 0, nL = 0;
    sv_dtype dt = SV_C64;
    size_t es = 8;
    int device = 0;
    cudaStream_t stream = nullptr;
    void *psi = nullptr;
    bool psi_owned = false;
    void *lam = nullptr;
    bool lam_owned = false;
    std::vector<int32_t> l2p;
    sv_options opt;
    uint64_t tick = 0;
    std::vector<std::unique_ptr<QsuEntry>> qsu;
    std::vector<std::unique_ptr<EvcEntry>> evc, hps;
    DevBuf params, coef, mats, part, slotval, opval, grad, scal, per_term, status;
    // forward bookkeeping for SV_FORWARD_DONE
    uint64_t last_qsu_key = 0;
    bool forward_valid = false;
    // forward checkpoints (options.checkpoint_every): copies of psi after
    // selected gate passes of the plan last applied, device or pinned host
    struct Ckpt { int pass; void *p; bool host; };
    std::vector<Ckpt> ckpts;
    uint64_t ckpt_key = 0;
    void drop_ckpts() {
        for (auto &c : ckpts) {
            if (c.host) cudaFreeHost(c.p);
            else cudaFree(c.p);
        }
        ckpts.clear();
        ckpt_key = 0;
    }
    // profiling: event pairs of launches not yet resolved
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    cudaEvent_t ev_get() {
        if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    size_t state_bytes() const { return ((size_t)1 << n) * es; }
};

struct sv_plan {
    int kind = 0;   // 0 QSU, 1 EVC
    QsuPlan q;
    EvcPlan e;
};

namespace {

void stats_clear(sv_stats *s) {
    if (s) memset(s, 0, sizeof(*s));
}

// Counts one launch of a kernel kind with its algorithmic bytes; with
// options.profile it brackets the launch with CUDA events on the stream.
struct Rec {
    sv_handle *h;
    sv_stats *st;
    int kind;
    cudaEvent_t a = nullptr;
    Rec(sv_handle *h_, sv_stats *st_, int kind_, double bytes) : h(h_), st(st_), kind(kind_) {
        if (st) {
            st->kernels[kind]++;
            st->bytes[kind] += bytes;
            st->launches++;
        }
        if (st && h->opt.profile) {
            a = h->ev_get();
            cudaEventRecord(a, h->stream);
        }
    }
    ~Rec() {
        if (a) {
            cudaEvent_t b = h->ev_get();
            cudaEventRecord(b, h->stream);
            h->pending.push_back({kind, a, b});
        }
    }
};

// Synchronise and add the timed launches into st->ms.
sv_status resolve_profile(sv_handle *h, sv_stats *st) {
    if (h->pending.empty()) return SV_OK;
    SV_CK(cudaStreamSynchronize(h->stream));
    for (auto &p : h->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        if (st) st->ms[p.kind] += ms;
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    h->pending.clear();
    return SV_OK;
}

sv_status ensure_psi(sv_handle *h) {
    if (h->psi) return SV_OK;
    SV_CK(cudaSetDevice(h->device));
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, h->state_bytes());
    if (e != cudaSuccess) return fail(SV_ENOMEM, std::string("state allocation: ") + cudaGetErrorString(e));
    h->psi = p;
    h->psi_owned = true;
    SV_CK(launch_set_basis(h->dt, h->stream, h->psi, h->state_bytes(), 0));
    return SV_OK;
}

sv_status ensure_lam(sv_handle *h) {
    if (h->lam) return SV_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, h->state_bytes());
    if (e != cudaSuccess) return fail(SV_ENOMEM, std::string("lambda allocation: ") + cudaGetErrorString(e));
    h->lam = p;
    h->lam_owned = true;
    return SV_OK;
}

bool identity(const std::vector<int32_t> &l2p) {
    for (size_t q = 0; q < l2p.size(); ++q)
        if (l2p[q] != (int32_t)q) return false;
    return true;
}

// Move the state (and lambda if given) from layout h->l2p to `to`.
sv_status relayout(sv_handle *h, const std::vector<int32_t> &to, bool with_lam, sv_stats *st) {
    if (to == h->l2p) return SV_OK;
    std::vector<std::vector<int32_t>> sets;
    permutation_swaps(h->l2p, to, sets);
    for (auto &s : sets) {
        {
            Rec r(h, st, SV_K_PERM, 2.0 * (double)h->state_bytes());
            SV_CK(launch_bitswap(h->dt, h->stream, h->psi, h->n, s.data(), (int)s.size() / 2, h->opt.blocks_per_sm));
        }
        if (with_lam) {
            Rec r(h, st, SV_K_PERM, 2.0 * (double)h->state_bytes());
            SV_CK(launch_bitswap(h->dt, h->stream, h->lam, h->n, s.data(), (int)s.size() / 2, h->opt.blocks_per_sm));
        }
    }
    h->l2p = to;
    return SV_OK;
}

uint64_t qsu_key(const sv_handle *h, const sv_gate *gates, size_t m, size_t np, sv_schedule sched) {
    uint64_t k = hash_bytes(gates, m * sizeof(sv_gate));
    k = hash_bytes(&np, sizeof(np), k);
    k = hash_bytes(&sched, sizeof(sched), k);
    k = hash_bytes(&h->opt, sizeof(h->opt), k);
    k = hash_bytes(h->l2p.data(), h->l2p.size() * sizeof(int32_t), k);
    return k;
}

// Greedy steps of Alg. 6 on the device (see k_alg6_step); buffers live for
// one plan.
struct Alg6Device {
    DevBuf xs, w, binom, best;
    cudaStream_t st = nullptr;
    int n = -1, k = -1;
    size_t nx = 0;
    ~Alg6Device() {
        if (st) cudaStreamDestroy(st);
        xs.release(); w.release(); binom.release(); best.release();
    }
    std::string step(const std::vector<uint64_t> &X, const std::vector<int32_t> &W, int n_, int k_, int64_t &rank,
                     int64_t &count) {
        auto cuerr = [](const char *what, cudaError_t e) { return std::string(what) + ": " + cudaGetErrorString(e); };
        cudaError_t e;
        if (!st && (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return cuerr("stream", e);
        std::vector<int64_t> B((size_t)(n_ + 1) * (k_ + 1), 0);
        for (int a = 0; a <= n_; ++a)
            for (int b = 0; b <= k_ && b <= a; ++b) {
                long double c = 1;
                for (int i = 1; i <= b; ++i) c = c * (a - b + i) / i;
                B[(size_t)a * (k_ + 1) + b] = (int64_t)(c + 0.5L);
            }
        const uint64_t ncand = (uint64_t)B[(size_t)n_ * (k_ + 1) + k_];
        if (ncand >= (1ull << 32)) return "Alg. 6 search space C(n, n_G) beyond 2^32";
        if (n_ != n || k_ != k) {
            if ((e = upload(binom, B, st)) != cudaSuccess) return cuerr("binomials", e);
            n = n_;
            k = k_;
        }
        if (X.size() != nx) {
            if ((e = upload(xs, X, st)) != cudaSuccess) return cuerr("supports", e);
            nx = X.size();
        }
        if ((e = upload(w, W, st)) != cudaSuccess) return cuerr("weights", e);
        if ((e = best.ensure(8)) != cudaSuccess) return cuerr("alloc", e);
        if ((e = cudaMemsetAsync(best.p, 0, 8, st)) != cudaSuccess) return cuerr("memset", e);
        if ((e = launch_alg6_step(st, xs.as<uint64_t>(), w.as<int32_t>(), (int)X.size(), n_, k_, binom.as<int64_t>(),
                                  ncand, (unsigned long long *)best.p)) != cudaSuccess)
            return cuerr("Alg. 6 kernel", e);
        unsigned long long key = 0;
        if ((e = cudaMemcpyAsync(&key, best.p, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuerr("copy", e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuerr("sync", e);
        count = (int64_t)(key >> 32);
        rank = (int64_t)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
        return "";
    }
};

bool alg6_on_device(int plan_device, int n, int g) {
    if (plan_device == 2) return false;
    if (plan_device == 1) return true;
    long double c = 1;
    for (int i = 1; i <= g; ++i) c = c * (n - g + i) / i;
    if (c < (long double)(1 << 19)) return false;
    int cnt = 0;
    return cudaGetDeviceCount(&cnt) == cudaSuccess && cnt > 0;
}

sv_status check_sched(sv_schedule s) {
    if (s != SV_SCHED_EAGER && s != SV_SCHED_LAZY && s != SV_SCHED_DIRECT && s != SV_SCHED_HIER &&
        s != SV_SCHED_LAZY_DIAG)
        return fail(SV_EINVAL, "bad schedule");
    return SV_OK;
}

sv_status get_qsu(sv_handle *h, const sv_gate *gates, size_t m, size_t np, sv_schedule sched, QsuEntry **out,
                  sv_stats *st) {
    SV_TRY(check_sched(sched));
    uint64_t key = qsu_key(h, gates, m, np, sched);
    ++h->tick;
    for (auto &e : h->qsu)
        if (e->key == key) {
            e->last_use = h->tick;
            *out = e.get();
            if (st) st->plan_cache_hit = 1;
            return SV_OK;
        }
    auto ent = std::make_unique<QsuEntry>();
    auto t0 = std::chrono::steady_clock::now();
    PlanOptions po = plan_options(h->opt);
    if (sched == SV_SCHED_HIER) po.hier_intra = h->opt.intra_bits;
    po.diag_exempt = sched == SV_SCHED_LAZY_DIAG;
    po.amp_bytes = h->dt == SV_C64 ? 8 : 16;              // the diagonal blocks' shared-memory budget
    std::string err = plan_qsu(h->n, sched == SV_SCHED_DIRECT ? 0 : h->g, gates, m, sched != SV_SCHED_EAGER, po,
                               h->l2p, ent->plan);
    if (!err.empty()) return fail(SV_EINVAL, "QSU plan: " + err);
    ent->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ent->key = key;
    ent->m = (int)m;
    ent->np = (int)np;
    for (auto &gp : ent->plan.passes) ent->args.push_back(gate_args(h->n, gp));
    SV_CK(upload(ent->ops, ent->plan.ops, h->stream));
    SV_CK(upload(ent->phases, ent->plan.phases, h->stream));
    SV_CK(upload(ent->steps, ent->plan.steps, h->stream));
    SV_CK(upload(ent->dblocks, ent->plan.dblocks, h->stream));
    SV_CK(upload(ent->dmembers, ent->plan.dmembers, h->stream));
    std::vector<int32_t> gparam(m);
    for (size_t i = 0; i < m; ++i) gparam[i] = gates[i].param;
    bool parametric_kind[8] = {true, true, false, true, true, false, false, false};
    for (size_t i = 0; i < m; ++i)
        if (!parametric_kind[gates[i].kind]) gparam[i] = -1;
    SV_CK(upload(ent->gparam, gparam, h->stream));
    // parameter -> pass operations (fixed order) for the gradient scatter
    std::vector<int32_t> off(np + 1, 0), idx;
    for (size_t o = 0; o < ent->plan.ops.size(); ++o) {
        int p = gparam[ent->plan.ops[o].gate];
        if (p >= 0) off[p + 1]++;
    }
    for (size_t p = 0; p < np; ++p) off[p + 1] += off[p];
    idx.resize(off[np]);
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (size_t o = 0; o < ent->plan.ops.size(); ++o) {
        int p = gparam[ent->plan.ops[o].gate];
        if (p >= 0) idx[fill[p]++] = (int32_t)o;
    }
    SV_CK(upload(ent->csr_off, off, h->stream));
    SV_CK(upload(ent->csr_idx, idx, h->stream));
    if (st) st->plan_ms = ent->plan_ms;
    ent->last_use = h->tick;
    if (h->qsu.size() >= kCacheSize) {
        auto it = std::min_element(h->qsu.begin(), h->qsu.end(),
                                   [](auto &a, auto &b) { return a->last_use < b->last_use; });
        SV_CK(cudaStreamSynchronize(h->stream));
        (*it)->release();
        h->qsu.erase(it);
    }
    *out = ent.get();
    h->qsu.push_back(std::move(ent));
    return SV_OK;
}

sv_status evc_entry_upload(sv_handle *h, EvcEntry *ent, const double *coeffs, size_t nterms) {
    std::vector<DevGroup> gs(ent->plan.groups.size());
    for (size_t i = 0; i < gs.size(); ++i) {
        const EvcGroup &g = ent->plan.groups[i];
        gs[i].x = g.x;
        gs[i].X = g.X;
        gs[i].s_begin = g.s_begin;
        gs[i].s_end = g.s_end;
        gs[i].parts = 0;
        for (int32_t q = g.s_begin; q < g.s_end; ++q) gs[i].parts |= 1 << (ent->plan.strings[q].nY & 1);
    }
    std::vector<DevString> ss(ent->plan.strings.size());
    for (size_t i = 0; i < ss.size(); ++i) {
        ss[i].z = ent->plan.strings[i].z;
        ss[i].coef = ent->plan.strings[i].coef;
        ss[i].nY = ent->plan.strings[i].nY;
        ss[i].bz = ent->plan.strings[i].bz;
    }
    SV_CK(upload(ent->groups, gs, h->stream));
    SV_CK(upload(ent->strings, ss, h->stream));
    SV_CK(upload(ent->term_slot, ent->plan.term_slot, h->stream));
    std::vector<double> c(coeffs, coeffs + nterms);
    SV_CK(upload(ent->coeffs, c, h->stream));
    for (auto &cp : ent->plan.passes) ent->args.push_back(coset_args(h->n, cp));
    return SV_OK;
}

void cache_insert(sv_handle *h, std::vector<std::unique_ptr<EvcEntry>> &cache, std::unique_ptr<EvcEntry> ent) {
    if (cache.size() >= kCacheSize) {
        auto it = std::min_element(cache.begin(), cache.end(),
                                   [](auto &a, auto &b) { return a->last_use < b->last_use; });
        cudaStreamSynchronize(h->stream);
        (*it)->release();
        cache.erase(it);
    }
    cache.push_back(std::move(ent));
}

sv_status check_paulis(const sv_handle *h, const sv_pauli *p, const double *c, size_t nterms) {
    const uint64_t lim = h->n >= 64 ? ~0ull : ((1ull << h->n) - 1);
    for (size_t t = 0; t < nterms; ++t) {
        if ((p[t].x & ~lim) || (p[t].z & ~lim)) return fail(SV_EINVAL, "Pauli mask beyond n qubits");
        if (c && !std::isfinite(c[t])) return fail(SV_EINVAL, "non-finite coefficient");
    }
    return SV_OK;
}

sv_status get_evc(sv_handle *h, const sv_pauli *p, const double *c, size_t nterms, sv_schedule sched, bool hpsi,
                  EvcEntry **out, sv_stats *st) {
    uint64_t key = hash_bytes(p, nterms * sizeof(sv_pauli));
    key = hash_bytes(c, nterms * sizeof(double), key);
    int flags = (int)sched | (hpsi ? 4 : 0);
    key = hash_bytes(&flags, sizeof(flags), key);
    key = hash_bytes(&h->opt, sizeof(h->opt), key);
    key = hash_bytes(h->l2p.data(), h->l2p.size() * sizeof(int32_t), key);
    auto &cache = hpsi ? h->hps : h->evc;
    ++h->tick;
    for (auto &e : cache)
        if (e->key == key) {
            e->last_use = h->tick;
            *out = e.get();
            if (st) st->plan_cache_hit = 1;
            return SV_OK;
        }
    auto ent = std::make_unique<EvcEntry>();
    auto t0 = std::chrono::steady_clock::now();
    PlanOptions po = plan_options(h->opt);
    Alg6Device a6;
    if (!hpsi && sched != SV_SCHED_DIRECT && alg6_on_device(h->opt.plan_device, h->n, h->g))
        po.alg6_step = [&](const std::vector<uint64_t> &X, const std::vector<int32_t> &W, int n_, int k_, int64_t &r,
                           int64_t &c) { return a6.step(X, W, n_, k_, r, c); };
    std::string err = (hpsi || sched == SV_SCHED_DIRECT)
                          ? plan_hpsi(h->n, p, c, nterms, po, h->l2p, ent->plan)
                          : plan_evc(h->n, h->g, p, c, nterms, sched != SV_SCHED_EAGER, po, h->l2p, ent->plan);
    if (!err.empty()) return fail(SV_EINVAL, std::string(hpsi ? "H|psi> plan: " : "EVC plan: ") + err);
    ent->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ent->key = key;
    ent->nterms = (int)nterms;
    SV_TRY(evc_entry_upload(h, ent.get(), c, nterms));
    if (st) st->plan_ms += ent->plan_ms;
    ent->last_use = h->tick;
    *out = ent.get();
    cache_insert(h, cache, std::move(ent));
    return SV_OK;
}

sv_status upload_params(sv_handle *h, QsuEntry *q, const double *params, size_t np, const double *mats,
                        size_t nmats, sv_stats *st) {
    for (size_t i = 0; i < np; ++i)
        if (!std::isfinite(params[i])) return fail(SV_EINVAL, "non-finite parameter");
    std::vector<double> pv(params, params + np);
    SV_CK(upload(h->params, pv, h->stream));
    SV_CK(h->coef.ensure(std::max<size_t>((size_t)q->m * h->es, 16)));   // (cos, sin) per gate
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_prep(h->dt, h->stream, q->gparam.as<int32_t>(), h->params.as<double>(), q->m, h->coef.p));
    }
    if (mats && nmats) {
        if (h->dt == SV_C64) {
            std::vector<float> mf(2 * nmats);
            for (size_t i = 0; i < 2 * nmats; ++i) mf[i] = (float)mats[i];
            SV_CK(upload(h->mats, mf, h->stream));
        } else {
            std::vector<double> md(mats, mats + 2 * nmats);
            SV_CK(upload(h->mats, md, h->stream));
        }
    } else {
        SV_CK(h->mats.ensure(16));
    }
    return SV_OK;
}

// Gate passes run 256-thread CTAs (two per SM); adjoint passes use
// options.threads (default 512: they hold two tiles and need more warps).
int gate_threads(const sv_handle *h) { return std::min(256, h->opt.threads > 0 ? h->opt.threads : 256); }
int adj_threads(const sv_handle *h) { return h->opt.threads > 0 ? h->opt.threads : 512; }

// Copy psi after gate pass `pass` into a checkpoint slot: device memory if
// available, else pinned host memory (the case where the state buffers do not
// all fit in HBM).
sv_status take_checkpoint(sv_handle *h, int pass, sv_stats *st) {
    void *p = nullptr;
    bool host = false;
    if (cudaMalloc(&p, h->state_bytes()) != cudaSuccess) {
        cudaGetLastError();
        host = true;
        if (cudaMallocHost(&p, h->state_bytes()) != cudaSuccess)
            return fail(SV_ENOMEM, "no room for a forward checkpoint on the device or the host");
    }
    h->ckpts.push_back({pass, p, host});
    Rec r(h, st, SV_K_PERM, 2.0 * (double)h->state_bytes());
    SV_CK(cudaMemcpyAsync(p, h->psi, h->state_bytes(), host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          h->stream));
    return SV_OK;
}

sv_status run_forward(sv_handle *h, QsuEntry *q, sv_stats *st) {
    const QsuPlan &P = q->plan;
    const int threads = gate_threads(h);
    h->drop_ckpts();
    size_t pi = 0;
    for (size_t t = 0; t < P.tiles.size(); ++t) {
        const Tile &T = P.tiles[t];
        if (!T.pairs.empty()) {
            const int s = (int)T.pairs.size() / 2;
            Rec r(h, st, SV_K_QR, 2.0 * (1.0 - std::ldexp(1.0, -s)) * (double)h->state_bytes());
            SV_CK(launch_bitswap(h->dt, h->stream, h->psi, h->n, T.pairs.data(), s, h->opt.blocks_per_sm));
        }
        for (; pi < P.passes.size() && P.passes[pi].tile == (int)t; ++pi) {
            const GatePassArgs &a = q->args[pi];
            int grid = gate_pass_grid(h->dt, a.k, a.nlow, a.op_end - a.op_begin, threads, h->opt.blocks_per_sm);
            uint64_t ntiles = 1ull << a.nout;
            if ((uint64_t)grid > ntiles) grid = (int)ntiles;
            if (a.ph_begin >= 0) {
                Rec r(h, st, SV_K_GATE, 2.0 * (double)h->state_bytes());
                const int rg = (int)std::min<uint64_t>(ntiles, (uint64_t)device_sms());
                SV_CK(launch_gate_reg(h->dt, h->stream, rg, h->psi, a, q->ops.as<DevOp>(), q->phases.as<Phase>(),
                                      q->steps.as<RegStep>(), h->coef.p, h->mats.p, q->dblocks.as<DiagBlock>(),
                                      q->dmembers.as<DiagMember>()));
            } else {
                Rec r(h, st, SV_K_GATE, 2.0 * (double)h->state_bytes());
                SV_CK(launch_gate_pass(h->dt, h->stream, grid, threads, h->psi, a, q->ops.as<DevOp>(), h->coef.p,
                                       h->mats.p));
            }
            const int c = h->opt.checkpoint_every;
            if (c > 0 && (int)(pi + 1) % c == 0 && pi + 1 < P.passes.size()) SV_TRY(take_checkpoint(h, (int)pi, st));
        }
    }
    if (h->opt.checkpoint_every > 0) h->ckpt_key = q->key;
    if (st) {
        st->qsu_tiles = (int32_t)P.tiles.size();
        st->qsu_qrs = P.nqr();
        st->qsu_passes = (int32_t)P.passes.size();
    }
    h->l2p = P.final_l2p;
    return SV_OK;
}

sv_status run_evc(sv_handle *h, EvcEntry *e, double *energy, double *per_term, sv_stats *st) {
    const EvcPlan &P = e->plan;
    const int nslots = (int)P.strings.size();
    int E = 1;
    for (auto &cp : P.passes) E = std::max(E, 1 << (cp.kl + cp.m));
    const int grid = coset_grid(h->dt, E, h->opt.blocks_per_sm, false);
    SV_CK(h->part.ensure((size_t)grid * std::max(nslots, 1) * sizeof(double)));
    SV_CK(h->slotval.ensure(std::max(nslots, 1) * sizeof(double)));
    SV_CK(h->scal.ensure(4 * sizeof(double)));
    SV_CK(h->per_term.ensure(std::max(e->nterms, 1) * sizeof(double)));
    for (size_t t = 0; t < P.tiles.size(); ++t) {
        const Tile &T = P.tiles[t];
        if (!T.pairs.empty()) {
            const int s = (int)T.pairs.size() / 2;
            Rec r(h, st, SV_K_QR, 2.0 * (1.0 - std::ldexp(1.0, -s)) * (double)h->state_bytes());
            SV_CK(launch_bitswap(h->dt, h->stream, h->psi, h->n, T.pairs.data(), s, h->opt.blocks_per_sm));
        }
        for (int pi = P.tile_pass_begin[t]; pi < P.tile_pass_end[t]; ++pi) {
            Rec r(h, st, SV_K_EVC, (double)h->state_bytes());
            SV_CK(launch_evc_pass(h->dt, h->stream, grid, h->psi, e->args[pi], e->groups.as<DevGroup>(),
                                  e->strings.as<DevString>(), h->part.as<double>(), nslots, h->status.as<int>(),
                                  (long long)h->opt.wait_limit));
        }
    }
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_reduce_rows(h->stream, h->part.as<double>(), grid, nslots, 0, nslots, h->slotval.as<double>()));
    }
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_energy(h->stream, h->slotval.as<double>(), e->term_slot.as<int32_t>(), e->coeffs.as<double>(),
                            e->nterms, h->per_term.as<double>(), h->scal.as<double>()));
    }
    if (st) {
        st->evc_tiles = (int32_t)P.tiles.size();
        st->evc_qrs = P.nqr();
        st->evc_passes = (int32_t)P.passes.size();
    }
    h->l2p = P.final_l2p;
    if (energy) SV_CK(cudaMemcpyAsync(energy, h->scal.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (per_term && e->nterms)
        SV_CK(cudaMemcpyAsync(per_term, h->per_term.p, e->nterms * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    return SV_OK;
}

// lambda = H psi; energy into h->scal[1] (device).
sv_status run_hpsi(sv_handle *h, EvcEntry *e, sv_stats *st) {
    const EvcPlan &P = e->plan;
    SV_TRY(ensure_lam(h));
    int E = 1;
    for (auto &cp : P.passes) E = std::max(E, 1 << (cp.kl + cp.m));
    const int grid = coset_grid(h->dt, E, h->opt.blocks_per_sm, true);
    SV_CK(h->part.ensure((size_t)grid * sizeof(double) + 64));
    SV_CK(h->scal.ensure(4 * sizeof(double)));
    const int np = (int)P.passes.size();
    if (np == 0) {
        SV_CK(cudaMemsetAsync(h->lam, 0, h->state_bytes(), h->stream));
        SV_CK(cudaMemsetAsync(h->scal.as<double>() + 1, 0, sizeof(double), h->stream));
        return SV_OK;
    }
    for (int pi = 0; pi < np; ++pi) {
        Rec r(h, st, SV_K_HPSI, (pi == 0 ? 2.0 : 3.0) * (double)h->state_bytes());
        SV_CK(launch_hpsi_pass(h->dt, h->stream, grid, h->psi, h->lam, e->args[pi], e->groups.as<DevGroup>(),
                               e->strings.as<DevString>(), pi == 0, pi == np - 1, h->part.as<double>(),
                               h->status.as<int>(), (long long)h->opt.wait_limit));
    }
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_reduce_rows(h->stream, h->part.as<double>(), grid, 1, 0, 1, h->scal.as<double>() + 1));
    }
    if (st) st->hpsi_passes = np;
    return SV_OK;
}

sv_status run_reverse(sv_handle *h, QsuEntry *q, sv_stats *st) {
    const QsuPlan &P = q->plan;
    const int threads = adj_threads(h);
    const int nops = (int)P.ops.size();
    int grid = 1;
    for (auto &a : q->args)
        grid = std::max(grid, adj_pass_grid(h->dt, a.k, a.nlow, a.op_end - a.op_begin, threads, h->opt.blocks_per_sm));
    SV_CK(h->part.ensure((size_t)grid * std::max(nops, 1) * sizeof(double)));
    SV_CK(h->opval.ensure(std::max(nops, 1) * sizeof(double)));
    SV_CK(h->grad.ensure(std::max(q->np, 1) * sizeof(double)));
    int pi = (int)P.passes.size() - 1;
    for (int t = (int)P.tiles.size() - 1; t >= 0; --t) {
        for (; pi >= 0 && P.passes[pi].tile == t; --pi) {
            const GatePassArgs &a = q->args[pi];
            if (h->ckpt_key == q->key)
                for (auto &c : h->ckpts)
                    if (c.pass == pi) {   // re-anchor psi at the forward value after this pass
                        Rec r(h, st, SV_K_PERM, 2.0 * (double)h->state_bytes());
                        SV_CK(cudaMemcpyAsync(h->psi, c.p, h->state_bytes(),
                                              c.host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
                    }
            Rec r(h, st, SV_K_ADJ, 4.0 * (double)h->state_bytes());
            if (a.ph_begin >= 0)
                SV_CK(launch_adj_reg(h->dt, h->stream, grid, h->psi, h->lam, a, q->ops.as<DevOp>(),
                                     q->phases.as<Phase>(), q->steps.as<RegStep>(), h->coef.p, h->mats.p,
                                     h->part.as<double>(), nops, q->dblocks.as<DiagBlock>(),
                                     q->dmembers.as<DiagMember>()));
            else
                SV_CK(launch_adj_pass(h->dt, h->stream, grid, threads, h->psi, h->lam, a, q->ops.as<DevOp>(),
                                      h->coef.p, h->mats.p, h->part.as<double>(), nops));
            if (st) st->adj_passes++;
        }
        const Tile &T = P.tiles[t];
        if (!T.pairs.empty()) {
            const int s = (int)T.pairs.size() / 2;
            const double qb = 2.0 * (1.0 - std::ldexp(1.0, -s)) * (double)h->state_bytes();
            {
                Rec r(h, st, SV_K_QR, qb);
                SV_CK(launch_bitswap(h->dt, h->stream, h->psi, h->n, T.pairs.data(), s, h->opt.blocks_per_sm));
            }
            {
                Rec r(h, st, SV_K_QR, qb);
                SV_CK(launch_bitswap(h->dt, h->stream, h->lam, h->n, T.pairs.data(), s, h->opt.blocks_per_sm));
            }
        }
    }
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_reduce_rows(h->stream, h->part.as<double>(), grid, nops, 0, nops, h->opval.as<double>()));
    }
    {
        Rec r(h, st, SV_K_AUX, 0.0);
        SV_CK(launch_scatter(h->stream, h->opval.as<double>(), q->csr_off.as<int32_t>(), q->csr_idx.as<int32_t>(),
                             q->np, h->grad.as<double>()));
    }
    h->l2p = P.init_l2p;
    return SV_OK;
}

sv_status check_handle(const sv_handle *h) {
    if (!h) return fail(SV_EINVAL, "null handle");
    return SV_OK;
}

// Device status word of the coset kernels (bounded waits): cleared before a
// call's kernels, read after its synchronisation.
sv_status status_reset(sv_handle *h) {
    SV_CK(h->status.ensure(sizeof(int)));
    SV_CK(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
    return SV_OK;
}
sv_status status_check(sv_handle *h) {
    int v = 0;
    SV_CK(cudaMemcpy(&v, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) return fail(SV_ETIMEOUT, "a device wait for a bulk copy expired");
    return SV_OK;
}

}  // namespace

namespace sv {
void set_last_error(const std::string &m) { g_err = m; }
}  // namespace sv

extern "C" {

void sv_options_default(sv_dtype dt, sv_options *o) {
    memset(o, 0, sizeof(*o));
    o->tile_bits = dt == SV_C64 ? 13 : 12;
    o->low_bits = 4;
    o->evc_low_bits = dt == SV_C64 ? 5 : 4;     // shortest run; passes stage 2^(5+8) = 8192 amplitudes
    o->evc_span = 8;
    o->pad_highest = 1;
    o->checkpoint_every = 0;
    o->threads = 512;
    o->blocks_per_sm = 0;
    o->wait_limit = 1 << 26;
}

const char *sv_last_error(void) { return g_err.c_str(); }
const char *sv_version(void) { return "libsv 0.1 (sm_103a)"; }

sv_status sv_create(int n, int g, sv_dtype dt, sv_handle **out) {
    if (!out) return fail(SV_EINVAL, "null output");
    if (n < 1 || n > kMaxQubits) return fail(SV_EINVAL, "n must be in [1, 40]");
    if (g < 0 || g > n - 4) {
        if (!(g == 0 && n < 4)) return fail(SV_EINVAL, "g must be in [0, n - 4]");
    }
    if (dt != SV_C64 && dt != SV_C128) return fail(SV_EINVAL, "bad dtype");
    auto *h = new sv_handle();
    h->n = n;
    h->g = g;
    h->nL = n - g;
    h->dt = dt;
    h->es = dt == SV_C64 ? 8 : 16;
    cudaGetDevice(&h->device);
    h->l2p.resize(n);
    for (int q = 0; q < n; ++q) h->l2p[q] = q;
    sv_options_default(dt, &h->opt);
    *out = h;
    return SV_OK;
}

void sv_destroy(sv_handle *h) {
    if (!h) return;
    if (h->stream || h->psi) cudaStreamSynchronize(h->stream);
    for (auto &e : h->qsu) e->release();
    for (auto &e : h->evc) e->release();
    for (auto &e : h->hps) e->release();
    for (DevBuf *b : {&h->params, &h->coef, &h->mats, &h->part, &h->slotval, &h->opval, &h->grad, &h->scal,
                      &h->per_term, &h->status})
        b->release();
    h->drop_ckpts();
    for (auto &p : h->pending) { h->ev_pool.push_back(p.a); h->ev_pool.push_back(p.b); }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->psi_owned && h->psi) cudaFree(h->psi);
    if (h->lam_owned && h->lam) cudaFree(h->lam);
    delete h;
}

sv_status sv_attach_state(sv_handle *h, void *p, size_t bytes) {
    SV_TRY(check_handle(h));
    if (!p || bytes < h->state_bytes()) return fail(SV_EINVAL, "state buffer too small");
    if ((uintptr_t)p % 256) return fail(SV_EINVAL, "state buffer must be 256-byte aligned");
    if (h->psi_owned && h->psi) cudaFree(h->psi);
    h->psi = p;
    h->psi_owned = false;
    h->forward_valid = false;
    return SV_OK;
}

sv_status sv_attach_buffer(sv_handle *h, void *p, size_t bytes) { return sv_attach_state(h, p, bytes); }

sv_status sv_attach_lambda(sv_handle *h, void *p, size_t bytes) {
    SV_TRY(check_handle(h));
    if (!p || bytes < h->state_bytes()) return fail(SV_EINVAL, "lambda buffer too small");
    if ((uintptr_t)p % 256) return fail(SV_EINVAL, "lambda buffer must be 256-byte aligned");
    if (h->lam_owned && h->lam) cudaFree(h->lam);
    h->lam = p;
    h->lam_owned = false;
    return SV_OK;
}

sv_status sv_set_stream(sv_handle *h, void *stream) {
    SV_TRY(check_handle(h));
    h->stream = (cudaStream_t)stream;
    return SV_OK;
}

sv_status sv_set_options(sv_handle *h, const sv_options *o) {
    SV_TRY(check_handle(h));
    if (!o) return fail(SV_EINVAL, "null options");
    sv_options d;
    sv_options_default(h->dt, &d);
    sv_options n = *o;
    if (n.tile_bits <= 0) n.tile_bits = d.tile_bits;
    if (n.low_bits <= 0) n.low_bits = d.low_bits;
    if (n.evc_low_bits <= 0) n.evc_low_bits = d.evc_low_bits;
    if (n.evc_span < 0) n.evc_span = d.evc_span;
    if (n.threads <= 0) n.threads = d.threads;
    if (n.wait_limit <= 0) n.wait_limit = d.wait_limit;
    const int maxstage = h->dt == SV_C64 ? 13 : 12;
    if (n.tile_bits > maxstage || n.tile_bits < 5) return fail(SV_EINVAL, "tile_bits must be in [5, 13] (c64) / [5, 12] (c128)");
    if (n.low_bits > n.tile_bits - 4 || n.low_bits < 1) return fail(SV_EINVAL, "low_bits must be in [1, tile_bits - 4]");
    if (n.evc_low_bits + n.evc_span > maxstage) return fail(SV_EINVAL, "evc_low_bits + evc_span too large");
    if (n.evc_span > kMaxSpan) return fail(SV_EINVAL, "evc_span > 10");
    if (n.threads % 32 || n.threads > 512) return fail(SV_EINVAL, "threads must be a multiple of 32, <= 512");
    if (n.fuse_max < 0) return fail(SV_EINVAL, "fuse_max must be >= 0");
    if (n.intra_bits < 0 || n.intra_bits > h->g) return fail(SV_EINVAL, "intra_bits must be in [0, g]");
    if (n.plan_device < 0 || n.plan_device > 2) return fail(SV_EINVAL, "plan_device must be 0, 1 or 2");
    h->opt = n;
    return SV_OK;
}

sv_status sv_synchronize(sv_handle *h) {
    SV_TRY(check_handle(h));
    SV_CK(cudaStreamSynchronize(h->stream));
    return SV_OK;
}

sv_status sv_get_options(const sv_handle *h, sv_options *o) {
    if (!h || !o) return fail(SV_EINVAL, "null argument");
    *o = h->opt;
    return SV_OK;
}

sv_status sv_reset_basis(sv_handle *h, uint64_t index) {
    SV_TRY(check_handle(h));
    if (h->n < 64 && (index >> h->n)) return fail(SV_EINVAL, "basis index beyond 2^n");
    SV_TRY(ensure_psi(h));
    SV_CK(launch_set_basis(h->dt, h->stream, h->psi, h->state_bytes(), index));
    for (int q = 0; q < h->n; ++q) h->l2p[q] = q;
    h->forward_valid = false;
    return SV_OK;
}

sv_status sv_set_state(sv_handle *h, const void *src, int src_is_device) {
    SV_TRY(check_handle(h));
    if (!src) return fail(SV_EINVAL, "null source");
    SV_TRY(ensure_psi(h));
    SV_CK(cudaMemcpyAsync(h->psi, src, h->state_bytes(),
                          src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    if (!src_is_device) SV_CK(cudaStreamSynchronize(h->stream));
    for (int q = 0; q < h->n; ++q) h->l2p[q] = q;
    h->forward_valid = false;
    return SV_OK;
}

sv_status sv_get_state(sv_handle *h, void *dst, int dst_is_device, int logical_order) {
    SV_TRY(check_handle(h));
    if (!dst) return fail(SV_EINVAL, "null destination");
    SV_TRY(ensure_psi(h));
    if (logical_order && !identity(h->l2p)) {
        std::vector<int32_t> id(h->n);
        for (int q = 0; q < h->n; ++q) id[q] = q;
        SV_TRY(relayout(h, id, false, nullptr));
        h->forward_valid = false;
    }
    SV_CK(cudaMemcpyAsync(dst, h->psi, h->state_bytes(),
                          dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    SV_CK(cudaStreamSynchronize(h->stream));
    return SV_OK;
}

sv_status sv_get_permutation(const sv_handle *h, int32_t *l2p) {
    if (!h || !l2p) return fail(SV_EINVAL, "null argument");
    std::copy(h->l2p.begin(), h->l2p.end(), l2p);
    return SV_OK;
}

sv_status sv_apply_circuit(sv_handle *h, const sv_gate *gates, size_t m, const double *params, size_t np,
                           const double *mats, size_t nmats, sv_schedule sched, sv_stats *st) {
    SV_TRY(check_handle(h));
    stats_clear(st);
    if (m && !gates) return fail(SV_EINVAL, "null gate list");
    if (np && !params) return fail(SV_EINVAL, "null params");
    std::string err = validate_gates(h->n, gates, m, np, mats ? nmats : 0);
    if (!err.empty()) return fail(SV_EINVAL, err);
    SV_TRY(ensure_psi(h));
    QsuEntry *q = nullptr;
    SV_TRY(get_qsu(h, gates, m, np, sched, &q, st));
    SV_TRY(upload_params(h, q, params, np, mats, nmats, st));
    SV_TRY(run_forward(h, q, st));
    h->last_qsu_key = q->key;
    h->forward_valid = true;
    SV_TRY(resolve_profile(h, st));
    return SV_OK;
}

sv_status sv_expect(sv_handle *h, const sv_pauli *paulis, const double *coeffs, size_t nterms, sv_schedule sched,
                    uint32_t flags, double *energy, double *per_term, sv_stats *st) {
    SV_TRY(check_handle(h));
    stats_clear(st);
    if (nterms && (!paulis || !coeffs)) return fail(SV_EINVAL, "null Pauli list");
    SV_TRY(check_paulis(h, paulis, coeffs, nterms));
    SV_TRY(ensure_psi(h));
    std::vector<int32_t> entry = h->l2p;
    if (nterms == 0) {
        if (energy) *energy = 0.0;
        return SV_OK;
    }
    EvcEntry *e = nullptr;
    SV_TRY(check_sched(sched));
    SV_TRY(get_evc(h, paulis, coeffs, nterms, sched, false, &e, st));
    SV_TRY(status_reset(h));
    SV_TRY(run_evc(h, e, energy, per_term, st));
    if (flags & SV_KEEP_LAYOUT) SV_TRY(relayout(h, entry, false, st));
    else if (h->l2p != entry) h->forward_valid = false;
    SV_CK(cudaStreamSynchronize(h->stream));
    SV_TRY(status_check(h));
    SV_TRY(resolve_profile(h, st));
    return SV_OK;
}

sv_status sv_apply_hamiltonian(sv_handle *h, const sv_pauli *paulis, const double *coeffs, size_t nterms,
                               void *dst, double *energy, sv_stats *st) {
    SV_TRY(check_handle(h));
    stats_clear(st);
    if (nterms && (!paulis || !coeffs)) return fail(SV_EINVAL, "null Pauli list");
    SV_TRY(check_paulis(h, paulis, coeffs, nterms));
    SV_TRY(ensure_psi(h));
    EvcEntry *e = nullptr;
    SV_TRY(get_evc(h, paulis, coeffs, nterms, SV_SCHED_LAZY, true, &e, st));
    SV_TRY(status_reset(h));
    SV_TRY(run_hpsi(h, e, st));
    if (dst) SV_CK(cudaMemcpyAsync(dst, h->lam, h->state_bytes(), cudaMemcpyDeviceToDevice, h->stream));
    if (energy) SV_CK(cudaMemcpyAsync(energy, h->scal.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SV_CK(cudaStreamSynchronize(h->stream));
    SV_TRY(status_check(h));
    SV_TRY(resolve_profile(h, st));
    return SV_OK;
}

sv_status sv_grad(sv_handle *h, const sv_gate *gates, size_t m, const double *params, size_t np,
                  const double *mats, size_t nmats, const sv_pauli *paulis, const double *coeffs, size_t nterms,
                  sv_schedule sched, uint32_t flags, double *energy, double *grad, sv_stats *st) {
    SV_TRY(check_handle(h));
    stats_clear(st);
    if (m && !gates) return fail(SV_EINVAL, "null gate list");
    if (np && !params) return fail(SV_EINVAL, "null params");
    if (nterms && (!paulis || !coeffs)) return fail(SV_EINVAL, "null Pauli list");
    std::string err = validate_gates(h->n, gates, m, np, mats ? nmats : 0);
    if (!err.empty()) return fail(SV_EINVAL, err);
    SV_TRY(check_paulis(h, paulis, coeffs, nterms));
    SV_TRY(ensure_psi(h));
    QsuEntry *q = nullptr;
    if (flags & SV_FORWARD_DONE) {
        if (!h->forward_valid) return fail(SV_ESTATE, "SV_FORWARD_DONE without a valid forward state");
        for (auto &e : h->qsu)
            if (e->key == h->last_qsu_key) q = e.get();
        if (!q) return fail(SV_ESTATE, "forward plan no longer cached");
        // the cached plan was made for these gates?
        uint64_t gk = qsu_key(h, gates, m, np, sched);
        (void)gk;
        if (q->m != (int)m || q->np != (int)np) return fail(SV_ESTATE, "SV_FORWARD_DONE with a different circuit");
        SV_TRY(upload_params(h, q, params, np, mats, nmats, st));
        SV_TRY(relayout(h, q->plan.final_l2p, false, st));
    } else {
        SV_TRY(get_qsu(h, gates, m, np, sched, &q, st));
        SV_TRY(upload_params(h, q, params, np, mats, nmats, st));
        SV_TRY(run_forward(h, q, st));
    }
    EvcEntry *e = nullptr;
    SV_TRY(get_evc(h, paulis, coeffs, nterms, SV_SCHED_LAZY, true, &e, st));
    SV_TRY(status_reset(h));
    SV_TRY(run_hpsi(h, e, st));
    SV_TRY(run_reverse(h, q, st));
    h->forward_valid = false;
    if (!h->ckpts.empty()) {
        SV_CK(cudaStreamSynchronize(h->stream));
        h->drop_ckpts();
    }
    if (grad && np) SV_CK(cudaMemcpyAsync(grad, h->grad.p, np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (energy) SV_CK(cudaMemcpyAsync(energy, h->scal.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SV_CK(cudaStreamSynchronize(h->stream));
    SV_TRY(status_check(h));
    SV_TRY(resolve_profile(h, st));
    return SV_OK;
}

sv_status sv_vqe_step(sv_handle *h, uint64_t init_index, const sv_gate *gates, size_t m, const double *params,
                      size_t np, const double *mats, size_t nmats, const sv_pauli *paulis, const double *coeffs,
                      size_t nterms, sv_schedule sched, double *energy, double *per_term, double *grad,
                      sv_stats *st) {
    SV_TRY(check_handle(h));
    sv_stats a, b, c, r;
    stats_clear(&r);
    {
        Rec rec(h, st ? &r : nullptr, SV_K_AUX, 0.0);
        SV_TRY(sv_reset_basis(h, init_index));
    }
    SV_TRY(resolve_profile(h, st ? &r : nullptr));
    SV_TRY(sv_apply_circuit(h, gates, m, params, np, mats, nmats, sched, st ? &a : nullptr));
    SV_TRY(sv_expect(h, paulis, coeffs, nterms, sched, SV_KEEP_LAYOUT, energy, per_term, st ? &b : nullptr));
    double e2 = 0;
    SV_TRY(sv_grad(h, gates, m, params, np, mats, nmats, paulis, coeffs, nterms, sched, SV_FORWARD_DONE, &e2, grad,
                   st ? &c : nullptr));
    if (st) {
        *st = a;
        st->evc_tiles = b.evc_tiles;
        st->evc_qrs = b.evc_qrs;
        st->evc_passes = b.evc_passes;
        st->hpsi_passes = c.hpsi_passes;
        st->adj_passes = c.adj_passes;
        st->launches = a.launches + b.launches + c.launches + r.launches;
        st->plan_cache_hit = a.plan_cache_hit && b.plan_cache_hit && c.plan_cache_hit;
        st->plan_ms = a.plan_ms + b.plan_ms + c.plan_ms;
        for (int k = 0; k < SV_K_COUNT; ++k) {
            st->kernels[k] = a.kernels[k] + b.kernels[k] + c.kernels[k] + r.kernels[k];
            st->bytes[k] = a.bytes[k] + b.bytes[k] + c.bytes[k] + r.bytes[k];
            st->ms[k] = a.ms[k] + b.ms[k] + c.ms[k] + r.ms[k];
        }
    }
    return SV_OK;
}

// ----------------------------------------------------------- host planning --

sv_status sv_plan_qsu(int n, int g, const sv_gate *gates, size_t m, sv_schedule sched, const sv_options *opt,
                      const int32_t *l2p_init, sv_plan **out) {
    if (!out || (m && !gates)) return fail(SV_EINVAL, "null argument");
    if (n < 1 || n > 63 || g < 0 || g > n - 1) return fail(SV_EINVAL, "bad n or g");
    size_t np = 0;
    for (size_t i = 0; i < m; ++i) np = std::max<size_t>(np, gates[i].param + 1);
    std::string err = validate_gates(n, gates, m, np, (size_t)-1);
    if (!err.empty()) return fail(SV_EINVAL, err);
    sv_options o;
    if (opt) o = *opt;
    else sv_options_default(SV_C64, &o);
    std::vector<int32_t> l2p(n);
    for (int q = 0; q < n; ++q) l2p[q] = l2p_init ? l2p_init[q] : q;
    auto *p = new sv_plan();
    p->kind = 0;
    SV_TRY(check_sched(sched));
    PlanOptions po = plan_options(o);
    if (sched == SV_SCHED_HIER) po.hier_intra = o.intra_bits;
    po.diag_exempt = sched == SV_SCHED_LAZY_DIAG;
    err = plan_qsu(n, sched == SV_SCHED_DIRECT ? 0 : g, gates, m, sched != SV_SCHED_EAGER, po, l2p, p->q);
    if (!err.empty()) {
        delete p;
        return fail(SV_EINVAL, err);
    }
    *out = p;
    return SV_OK;
}

sv_status sv_plan_evc(int n, int g, const sv_pauli *paulis, size_t nterms, sv_schedule sched, const sv_options *opt,
                      const int32_t *l2p_init, sv_plan **out) {
    if (!out || (nterms && !paulis)) return fail(SV_EINVAL, "null argument");
    if (n < 1 || n > 63 || g < 0 || g > n - 1) return fail(SV_EINVAL, "bad n or g");
    sv_options o;
    if (opt) o = *opt;
    else sv_options_default(SV_C64, &o);
    std::vector<int32_t> l2p(n);
    for (int q = 0; q < n; ++q) l2p[q] = l2p_init ? l2p_init[q] : q;
    std::vector<double> ones(nterms, 1.0);
    auto *p = new sv_plan();
    p->kind = 1;
    SV_TRY(check_sched(sched));
    PlanOptions po = plan_options(o);
    Alg6Device a6;
    if (sched != SV_SCHED_DIRECT && alg6_on_device(o.plan_device, n, g))
        po.alg6_step = [&](const std::vector<uint64_t> &X, const std::vector<int32_t> &W, int n_, int k_, int64_t &r,
                           int64_t &c) { return a6.step(X, W, n_, k_, r, c); };
    std::string err = sched == SV_SCHED_DIRECT
                          ? plan_hpsi(n, paulis, ones.data(), nterms, po, l2p, p->e)
                          : plan_evc(n, g, paulis, ones.data(), nterms, sched != SV_SCHED_EAGER, po, l2p, p->e);
    if (!err.empty()) {
        delete p;
        return fail(SV_EINVAL, err);
    }
    *out = p;
    return SV_OK;
}

sv_status sv_plan_info(const sv_plan *p, int32_t *ntiles, int32_t *nops, int32_t *npasses) {
    if (!p) return fail(SV_EINVAL, "null plan");
    const std::vector<Tile> &T = p->kind == 0 ? p->q.tiles : p->e.tiles;
    if (ntiles) *ntiles = (int32_t)T.size();
    if (nops) *nops = (int32_t)(p->kind == 0 ? p->q.order.size() : p->e.order.size());
    if (npasses) *npasses = (int32_t)(p->kind == 0 ? p->q.passes.size() : p->e.passes.size());
    return SV_OK;
}

sv_status sv_plan_order(const sv_plan *p, int32_t *order) {
    if (!p || !order) return fail(SV_EINVAL, "null argument");
    const std::vector<int32_t> &o = p->kind == 0 ? p->q.order : p->e.order;
    std::copy(o.begin(), o.end(), order);
    return SV_OK;
}

sv_status sv_plan_tile(const sv_plan *p, int32_t t, int32_t *begin, int32_t *end, uint64_t *local_mask,
                       int32_t *npairs, int32_t *pairs, int32_t *l2p) {
    if (!p) return fail(SV_EINVAL, "null plan");
    const std::vector<Tile> &T = p->kind == 0 ? p->q.tiles : p->e.tiles;
    if (t < 0 || t >= (int32_t)T.size()) return fail(SV_EINVAL, "tile index out of range");
    const Tile &x = T[t];
    if (begin) *begin = x.begin;
    if (end) *end = x.end;
    if (local_mask) *local_mask = x.local_mask;
    if (npairs) *npairs = (int32_t)x.pairs.size() / 2;
    if (pairs) std::copy(x.pairs.begin(), x.pairs.end(), pairs);
    if (l2p) std::copy(x.l2p.begin(), x.l2p.end(), l2p);
    return SV_OK;
}

sv_status sv_plan_tile_intra(const sv_plan *p, int32_t t, uint64_t *intra_mask) {
    if (!p || !intra_mask) return fail(SV_EINVAL, "null argument");
    const std::vector<Tile> &tiles = p->kind == 0 ? p->q.tiles : p->e.tiles;
    if (t < 0 || t >= (int32_t)tiles.size()) return fail(SV_EINVAL, "tile index out of range");
    *intra_mask = tiles[t].intra_mask;
    return SV_OK;
}

sv_status sv_plan_pass(const sv_plan *p, int32_t i, int32_t *tile, uint64_t *bits, int32_t *nops, int32_t *ops) {
    if (!p || p->kind != 0) return fail(SV_EINVAL, "not a QSU plan");
    if (i < 0 || i >= (int32_t)p->q.passes.size()) return fail(SV_EINVAL, "pass index out of range");
    const GatePass &gp = p->q.passes[i];
    if (tile) *tile = gp.tile;
    if (bits) *bits = gp.bits;
    if (nops) *nops = gp.op_end - gp.op_begin;
    if (ops)
        for (int o = gp.op_begin; o < gp.op_end; ++o) ops[o - gp.op_begin] = p->q.ops[o].gate;
    return SV_OK;
}

void sv_plan_free(sv_plan *p) { delete p; }

sv_status sv_batch_run(int n, sv_dtype dt, int batch, const sv_gate *gates, const int32_t *gate_off,
                       const double *params, const int32_t *param_off, const sv_pauli *paulis, const double *coeffs,
                       size_t nterms, uint64_t init_index, const sv_options *opt, void *stream, double *energies,
                       double *grads, double *times_ns, sv_stats *st) {
    stats_clear(st);
    if (n < 4 || n > 20) return fail(SV_EINVAL, "sv_batch_run: n must be in [4, 20]");
    if (dt != SV_C64 && dt != SV_C128) return fail(SV_EINVAL, "bad dtype");
    if (batch < 1 || !gates || !gate_off || !param_off || !energies) return fail(SV_EINVAL, "null argument");
    if ((nterms && (!paulis || !coeffs)) || (init_index >> n)) return fail(SV_EINVAL, "bad Hamiltonian or init");
    const uint64_t lim = (1ull << n) - 1;
    for (size_t t = 0; t < nterms; ++t) {
        if ((paulis[t].x & ~lim) || (paulis[t].z & ~lim)) return fail(SV_EINVAL, "Pauli mask beyond n qubits");
        if (!std::isfinite(coeffs[t])) return fail(SV_EINVAL, "non-finite coefficient");
    }
    sv_options o;
    if (opt) o = *opt;
    else sv_options_default(dt, &o);
    sv_options d;
    sv_options_default(dt, &d);
    // the kernel stages 2^tile_bits amplitudes per buffer; H|psi> coset
    // passes stage at most as many
    if (o.tile_bits <= 0) o.tile_bits = d.tile_bits;
    if (o.threads <= 0) o.threads = d.threads;
    if (o.low_bits <= 0) o.low_bits = d.low_bits;
    if (o.fuse_max < 0) return fail(SV_EINVAL, "fuse_max must be >= 0");
    if (!batch_supported(dt, o.tile_bits, o.threads))
        return fail(SV_EINVAL, "sv_batch_run: (tile_bits, threads) must give 2^tile_bits / threads in {4, 8, 16}, "
                               "tile_bits in [10, 13] (c64) / [10, 12] (c128), threads 256 or 512");
    if (o.low_bits > o.tile_bits - 4 || o.low_bits < 1) return fail(SV_EINVAL, "low_bits must be in [1, tile_bits - 4]");
    o.evc_low_bits = d.evc_low_bits;
    o.evc_span = std::min(d.evc_span, o.tile_bits - o.evc_low_bits);
    const int kmax = o.tile_bits;
    const int hio = std::max(8, kmax - o.low_bits);
    PlanOptions po = plan_options(o);
    po.max_diag = 0;                     // the batched kernel applies RZ / CZ one by one
    po.reg_pairs = false;                // and runs register phases of RY / RZ / CZ / 1-qubit matrices only
    std::vector<int32_t> l2p(n);
    for (int q = 0; q < n; ++q) l2p[q] = q;
    // one plan per distinct circuit
    std::vector<int32_t> state_plan(batch), plan_pass_off{0}, plan_op_off{0}, gparam;
    std::vector<GatePassArgs> passes;
    std::vector<Phase> phases;
    std::vector<DevOp> ops;
    std::vector<uint64_t> plan_keys;
    std::vector<int32_t> gsize(batch);
    auto t0 = std::chrono::steady_clock::now();
    for (int b = 0; b < batch; ++b) {
        const int gb = gate_off[b], ge = gate_off[b + 1];
        const int pb = param_off[b], pe = param_off[b + 1];
        if (ge < gb || pe < pb) return fail(SV_EINVAL, "offsets must be non-decreasing");
        const size_t m = (size_t)(ge - gb), np = (size_t)(pe - pb);
        if ((int)m > batch_max_gates()) return fail(SV_EINVAL, "sv_batch_run: more than 1024 gates in a state");
        std::string err = validate_gates(n, gates + gb, m, np, 0);
        if (!err.empty()) return fail(SV_EINVAL, "state " + std::to_string(b) + ": " + err);
        for (size_t i = 0; i < np; ++i)
            if (!std::isfinite(params[pb + i])) return fail(SV_EINVAL, "non-finite parameter");
        for (size_t i = 0; i < m; ++i) {
            const int k = gates[gb + i].kind;
            gparam.push_back((k == SV_RY || k == SV_RZ || k == SV_GIVENS || k == SV_DEXC) ? gates[gb + i].param : -1);
        }
        gsize[b] = (int)m;
        const uint64_t key = hash_bytes(gates + gb, m * sizeof(sv_gate));
        int pi = -1;
        for (size_t k = 0; k < plan_keys.size(); ++k)
            if (plan_keys[k] == key) pi = (int)k;
        if (pi < 0) {
            QsuPlan P;
            err = plan_qsu(n, 0, gates + gb, m, true, po, l2p, P);
            if (!err.empty()) return fail(SV_EINVAL, "state " + std::to_string(b) + ": " + err);
            if ((int)P.ops.size() > batch_max_ops()) return fail(SV_EINVAL, "sv_batch_run: more than 512 gates in a state");
            const int obase = (int)ops.size();
            const int pbase = (int)phases.size();
            for (auto &gp : P.passes) {
                GatePassArgs a = gate_args(n, gp);
                a.op_begin += obase;
                a.op_end += obase;
                if (a.ph_begin >= 0) {
                    a.ph_begin += pbase;
                    a.ph_end += pbase;
                }
                a.db_begin = a.db_end = 0;
                passes.push_back(a);
            }
            for (Phase f : P.phases) {
                f.op_begin += obase;
                f.op_end += obase;
                phases.push_back(f);
            }
            ops.insert(ops.end(), P.ops.begin(), P.ops.end());
            plan_pass_off.push_back((int32_t)passes.size());
            plan_op_off.push_back((int32_t)ops.size());
            pi = (int)plan_keys.size();
            plan_keys.push_back(key);
        }
        state_plan[b] = pi;
    }
    EvcPlan H;
    std::string err = plan_hpsi(n, paulis, coeffs, nterms, po, l2p, H);
    if (!err.empty()) return fail(SV_EINVAL, "H|psi> plan: " + err);
    std::vector<CosetArgs> hp;
    for (auto &cp : H.passes) hp.push_back(coset_args(n, cp));
    std::vector<DevGroup> gs(H.groups.size());
    for (size_t i = 0; i < gs.size(); ++i) {
        gs[i].x = H.groups[i].x;
        gs[i].X = H.groups[i].X;
        gs[i].s_begin = H.groups[i].s_begin;
        gs[i].s_end = H.groups[i].s_end;
        gs[i].parts = 0;
        for (int32_t q = H.groups[i].s_begin; q < H.groups[i].s_end; ++q) gs[i].parts |= 1 << (H.strings[q].nY & 1);
    }
    std::vector<DevString> ss(H.strings.size());
    for (size_t i = 0; i < ss.size(); ++i) {
        ss[i].z = H.strings[i].z;
        ss[i].coef = H.strings[i].coef;
        ss[i].nY = H.strings[i].nY;
        ss[i].bz = H.strings[i].bz;
    }
    std::vector<int32_t> order(batch);
    for (int b = 0; b < batch; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return gsize[x] > gsize[y]; });
    if (st) st->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

    cudaStream_t s0 = (cudaStream_t)stream;
    const int threads = o.threads;
    const int occ = batch_occupancy(dt, kmax, hio, threads);
    if (occ < 1) return fail(SV_EINVAL, "sv_batch_run: the batched kernel does not fit an SM with these options");
    const int grid = std::min(batch, device_sms() * occ);
    const size_t es = dt == SV_C64 ? 8 : 16;
    std::vector<DevBuf> bufs(17);
    auto up = [&](int i, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t e = bufs[i].ensure(std::max<size_t>(bytes, 16));
        if (e != cudaSuccess || !bytes) return e;
        return cudaMemcpyAsync(bufs[i].p, src, bytes, cudaMemcpyHostToDevice, s0);
    };
    auto release = [&]() {
        cudaStreamSynchronize(s0);
        for (auto &b : bufs) b.release();
    };
    const size_t nparams = (size_t)param_off[batch];
#define SV_BCK(call)                                                                                  \
    do {                                                                                              \
        cudaError_t _e = (call);                                                                      \
        if (_e != cudaSuccess) {                                                                      \
            release();                                                                                \
            return fail(SV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));                \
        }                                                                                             \
    } while (0)
    SV_BCK(up(0, passes.data(), passes.size() * sizeof(GatePassArgs)));
    SV_BCK(up(1, plan_pass_off.data(), plan_pass_off.size() * 4));
    SV_BCK(up(2, ops.data(), ops.size() * sizeof(DevOp)));
    SV_BCK(up(3, plan_op_off.data(), plan_op_off.size() * 4));
    SV_BCK(up(4, state_plan.data(), batch * 4));
    SV_BCK(up(5, order.data(), batch * 4));
    SV_BCK(up(6, gate_off, (batch + 1) * 4));
    SV_BCK(up(7, gparam.data(), gparam.size() * 4));
    SV_BCK(up(8, param_off, (batch + 1) * 4));
    SV_BCK(up(9, params, nparams * 8));
    SV_BCK(up(10, hp.data(), hp.size() * sizeof(CosetArgs)));
    SV_BCK(up(11, gs.data(), gs.size() * sizeof(DevGroup)));
    SV_BCK(up(12, ss.data(), ss.size() * sizeof(DevString)));
    SV_BCK(up(16, phases.data(), phases.size() * sizeof(Phase)));
    SV_BCK(bufs[13].ensure((size_t)grid * 2 * ((size_t)1 << n) * es));
    SV_BCK(bufs[14].ensure((batch + nparams + 2 * (size_t)batch) * 8 + 64));
    double *d_energy = bufs[14].as<double>();
    double *d_grads = d_energy + batch;
    unsigned long long *d_t = (unsigned long long *)(d_grads + nparams);
    SV_BCK(bufs[15].ensure(sizeof(int)));
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.nstates = batch;
    a.nhpass = (int)hp.size();
    a.kmax = kmax;
    a.hio = hio;
    a.init_index = init_index;
    a.passes = bufs[0].as<GatePassArgs>();
    a.phases = bufs[16].as<Phase>();
    a.plan_pass_off = bufs[1].as<int32_t>();
    a.ops = bufs[2].as<DevOp>();
    a.plan_op_off = bufs[3].as<int32_t>();
    a.state_plan = bufs[4].as<int32_t>();
    a.order = bufs[5].as<int32_t>();
    a.gate_off = bufs[6].as<int32_t>();
    a.gparam = bufs[7].as<int32_t>();
    a.param_off = bufs[8].as<int32_t>();
    a.params = bufs[9].as<double>();
    a.hpass = bufs[10].as<CosetArgs>();
    a.groups = bufs[11].as<DevGroup>();
    a.strs = bufs[12].as<DevString>();
    a.work = bufs[13].p;
    a.energies = d_energy;
    a.grads = d_grads;
    a.t_start = d_t;
    a.t_end = d_t + batch;
    a.counter = bufs[15].as<int>();
    // one graph: reset the work counter, then the persistent launch
    SV_BCK(cudaStreamSynchronize(s0));
    cudaStream_t cs = nullptr;
    SV_BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a.counter, 0, sizeof(int), cs);
    if (ce == cudaSuccess) ce = launch_batch(dt, cs, grid, threads, a);
    cudaError_t ce2 = cudaStreamEndCapture(cs, &graph);
    if (ce == cudaSuccess) ce = ce2;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, cs);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, cs);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, cs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    float ms = 0.f;
    if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
        release();
        return fail(SV_ECUDA, std::string("batched launch: ") + cudaGetErrorString(ce));
    }
    std::vector<unsigned long long> tt(2 * (size_t)batch);
    SV_BCK(cudaMemcpy(energies, d_energy, batch * 8, cudaMemcpyDeviceToHost));
    if (grads && nparams) SV_BCK(cudaMemcpy(grads, d_grads, nparams * 8, cudaMemcpyDeviceToHost));
    SV_BCK(cudaMemcpy(tt.data(), d_t, 2 * (size_t)batch * 8, cudaMemcpyDeviceToHost));
    if (times_ns) {
        unsigned long long t_min = ~0ull;
        for (int b = 0; b < batch; ++b) t_min = std::min(t_min, tt[b]);
        for (int b = 0; b < batch; ++b) {
            times_ns[2 * b] = (double)(tt[b] - t_min);
            times_ns[2 * b + 1] = (double)(tt[batch + b] - t_min);
        }
    }
    if (st) {
        st->launches = 1;
        st->kernels[SV_K_BATCH] = 1;
        st->ms[SV_K_BATCH] = ms;
        st->qsu_passes = (int32_t)passes.size();
        st->hpsi_passes = (int32_t)hp.size();
    }
    release();
#undef SV_BCK
    return SV_OK;
}

}  // extern "C"
