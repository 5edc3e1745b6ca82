// Autotuner for the implementation parameters the paper leaves open: the
// size 2^k of a gate pass's staged tile (tile_bits), the fusion depth (gate
// operations per pass, fuse_max), the shape of the coset passes of the
// expectation and H|psi> kernels (evc_low_bits, evc_span), and for the
// batched kernel its CTA size.  None of them changes a result beyond
// floating-point rounding order; they change HBM passes, shared-memory
// footprint and occupancy.
//
// Search: coordinate by coordinate from the starting options (tile size,
// then fusion depth, then coset shape), keeping a candidate only when it is
// faster.  Every candidate runs once untimed (planning, plan caches) and then
// `reps` times timed; the minimum counts.  Only the public C ABI is used.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "sv.h"

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Step {
    sv_handle *h;
    uint64_t init;
    const sv_gate *gates;
    size_t m;
    const double *params;
    size_t np;
    const double *mats;
    size_t nmats;
    const sv_pauli *paulis;
    const double *coeffs;
    size_t nterms;
    sv_schedule sched;
    std::vector<double> grad;

    sv_status run() {
        if (nterms) {
            double e = 0;
            return sv_vqe_step(h, init, gates, m, params, np, mats, nmats, paulis, coeffs, nterms, sched, &e, nullptr,
                               grad.data(), nullptr);
        }
        sv_status s = sv_reset_basis(h, init);
        if (s == SV_OK) s = sv_apply_circuit(h, gates, m, params, np, mats, nmats, sched, nullptr);
        if (s == SV_OK) s = sv_synchronize(h);
        return s;
    }

    // minimum over reps of the step's wall time with options o; < 0: o rejected
    sv_status time(const sv_options &o, int reps, double *ms) {
        *ms = -1.0;
        if (sv_set_options(h, &o) != SV_OK) return SV_OK;     // not a valid candidate for this handle
        sv_status s = run();
        if (s != SV_OK) return s;
        double best = 1e300;
        for (int r = 0; r < reps; ++r) {
            const double t0 = now_ms();
            s = run();
            if (s != SV_OK) return s;
            best = std::min(best, now_ms() - t0);
        }
        *ms = best;
        return SV_OK;
    }
};

bool same(const sv_options &a, const sv_options &b) { return memcmp(&a, &b, sizeof(a)) == 0; }

}  // namespace

extern "C" sv_status sv_autotune(sv_handle *h, uint64_t init_index, const sv_gate *gates, size_t m,
                                 const double *params, size_t np, const double *mats, size_t nmats,
                                 const sv_pauli *paulis, const double *coeffs, size_t nterms, sv_schedule sched,
                                 int reps, sv_options *best_out, double *best_ms) {
    if (!h || reps < 1) return SV_EINVAL;
    sv_options start;
    sv_status s = sv_get_options(h, &start);
    if (s != SV_OK) return s;
    Step st{h, init_index, gates, m, params, np, mats, nmats, paulis, coeffs, nterms, sched, std::vector<double>(np + 1)};
    sv_options best = start;
    double tbest = 0;
    s = st.time(best, reps, &tbest);
    if (s != SV_OK) return s;
    if (tbest < 0) return SV_EINVAL;
    std::vector<sv_options> tried{best};
    auto consider = [&](const sv_options &c) -> sv_status {
        for (auto &t : tried)
            if (same(t, c)) return SV_OK;
        tried.push_back(c);
        double t = 0;
        sv_status r = st.time(c, reps, &t);
        if (r != SV_OK) return r;
        if (t >= 0 && t < tbest) {
            tbest = t;
            best = c;
        }
        return SV_OK;
    };
    // 1. staged tile size k (largest first)
    const sv_options base = best;
    for (int k = base.tile_bits + 1; k >= 8; --k) {
        sv_options c = base;
        c.tile_bits = k;
        if (c.low_bits > k - 4) c.low_bits = k - 4;
        if ((s = consider(c)) != SV_OK) break;
    }
    // 2. fusion depth
    if (s == SV_OK) {
        const sv_options b2 = best;
        for (int f : {0, 64, 16, 4}) {
            sv_options c = b2;
            c.fuse_max = f;
            if ((s = consider(c)) != SV_OK) break;
        }
    }
    // 3. coset pass shape (only timed when the step evaluates strings)
    if (s == SV_OK && nterms) {
        const sv_options b3 = best;
        const int shapes[][2] = {{5, 8}, {4, 9}, {3, 10}, {4, 8}, {6, 7}, {5, 7}, {7, 6}};
        for (auto &sh : shapes) {
            sv_options c = b3;
            c.evc_low_bits = sh[0];
            c.evc_span = sh[1];
            if ((s = consider(c)) != SV_OK) break;
        }
    }
    // leave the handle on the fastest options, also after a failed candidate
    sv_status s2 = sv_set_options(h, &best);
    if (s != SV_OK) return s;
    if (s2 != SV_OK) return s2;
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = tbest;
    return SV_OK;
}

extern "C" sv_status sv_batch_autotune(int n, sv_dtype dt, int batch, const sv_gate *gates, const int32_t *gate_off,
                                       const double *params, const int32_t *param_off, const sv_pauli *paulis,
                                       const double *coeffs, size_t nterms, uint64_t init_index,
                                       const sv_options *start, void *stream, int reps, sv_options *best_out,
                                       double *best_ms) {
    if (batch < 1 || !gate_off || !param_off || reps < 1) return SV_EINVAL;
    sv_options base;
    if (start) base = *start;
    else sv_options_default(dt, &base);
    if (base.tile_bits <= 0 || base.threads <= 0) {
        sv_options d;
        sv_options_default(dt, &d);
        if (base.tile_bits <= 0) base.tile_bits = d.tile_bits;
        if (base.threads <= 0) base.threads = d.threads;
        if (base.low_bits <= 0) base.low_bits = d.low_bits;
    }
    std::vector<double> energies(batch), grads((size_t)param_off[batch] + 1);
    // device time of the batched launch (CUDA events around the graph launch)
    auto time = [&](const sv_options &o, double *ms) -> sv_status {
        *ms = -1.0;
        sv_stats stt;
        double best = 1e300;
        for (int r = 0; r <= reps; ++r) {
            sv_status s = sv_batch_run(n, dt, batch, gates, gate_off, params, param_off, paulis, coeffs, nterms,
                                       init_index, &o, stream, energies.data(), grads.data(), nullptr, &stt);
            if (s == SV_EINVAL) return SV_OK;        // not a valid candidate
            if (s != SV_OK) return s;
            if (r > 0) best = std::min(best, stt.ms[SV_K_BATCH]);
        }
        *ms = best;
        return SV_OK;
    };
    sv_options best = base;
    double tbest = 0;
    sv_status s = time(best, &tbest);
    if (s != SV_OK) return s;
    if (tbest < 0) return SV_EINVAL;
    std::vector<sv_options> tried{best};
    auto consider = [&](const sv_options &c) -> sv_status {
        for (auto &t : tried)
            if (same(t, c)) return SV_OK;
        tried.push_back(c);
        double t = 0;
        sv_status r = time(c, &t);
        if (r != SV_OK) return r;
        if (t >= 0 && t < tbest) {
            tbest = t;
            best = c;
        }
        return SV_OK;
    };
    // 1. (k, CTA size) pairs the batched kernel is built for
    const sv_options b1 = best;
    for (int k = 13; k >= 10 && s == SV_OK; --k)
        for (int th : {512, 256}) {
            sv_options c = b1;
            c.tile_bits = k;
            c.threads = th;
            if (c.low_bits > k - 4) c.low_bits = k - 4;
            if ((s = consider(c)) != SV_OK) break;
        }
    // 2. fusion depth
    if (s == SV_OK) {
        const sv_options b2 = best;
        for (int f : {0, 64, 16}) {
            sv_options c = b2;
            c.fuse_max = f;
            if ((s = consider(c)) != SV_OK) break;
        }
    }
    if (s != SV_OK) return s;
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = tbest;
    return SV_OK;
}
