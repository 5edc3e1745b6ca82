/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
 * its reference arm) may load this library.  The product path never does.
 *
 * Plain, slow, obviously correct FP64 state-vector simulator:
 *   - the state vector of Eq. (sv): 2^n complex amplitudes, qubit q <-> index
 *     bit q (Sec. III, "least and most significant bits ... qubits 0 and n-1");
 *   - QSU as the ordered gate product of Eq. (update_sv_gate), applied gate by
 *     gate in the GIVEN order, never reordered, never permuted;
 *   - every gate applied as its dense 2^k x 2^k matrix on its k targets;
 *   - EVC of Eq. (evc): <psi|P|psi> as a plain sum over basis states, with
 *     P's action taken letter by letter from the Pauli matrices of
 *     Eq. (pauli_matrix).
 *
 * Gate conventions (the paper never defines GateFabric's gates; these are the
 * readings the repository documents): U = exp(-i theta G / 2) with
 *   RY: G = Y;  RZ: G = Z;  CZ = diag(1,1,1,-1);
 *   GIVENS(phi) on (a,b): G = Y on span{|a=1,b=0>, |a=0,b=1>}, so
 *     |10> -> c|10> + s|01>,  |01> -> -s|10> + c|01>;
 *   DEXC(theta) on (q0..q3): G = Y on span{|q0=q1=1,q2=q3=0>, |q2=q3=1,q0=q1=0>};
 *   MAT1/MAT2/MAT4: caller matrix, row-major, complex interleaved.
 * Matrix index convention: local index j = sum_t bit(b, targets[t]) << t.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_RY = 0, K_RZ = 1, K_CZ = 2, K_GIVENS = 3, K_DEXC = 4, K_MAT1 = 5, K_MAT2 = 6, K_MAT4 = 7 };

static int gate_nq(int kind) {
    switch (kind) {
    case K_RY: case K_RZ: case K_MAT1: return 1;
    case K_CZ: case K_GIVENS: case K_MAT2: return 2;
    case K_DEXC: case K_MAT4: return 4;
    default: return -1;
    }
}

/* Build the dense matrix of one gate (row-major, re/im interleaved, dim^2). */
static int build_matrix(int kind, double theta, const double *mat, int inverse, double *u) {
    int nq = gate_nq(kind);
    if (nq < 0) return -1;
    int dim = 1 << nq;
    memset(u, 0, sizeof(double) * 2 * dim * dim);
    for (int i = 0; i < dim; ++i) u[2 * (i * dim + i)] = 1.0;
    double c = cos(0.5 * theta), s = sin(0.5 * theta);
    switch (kind) {
    case K_RY:
        u[2 * 0] = c;  u[2 * 1] = -s;
        u[2 * 2] = s;  u[2 * 3] = c;
        break;
    case K_RZ:
        /* diag(e^{-i theta/2}, e^{+i theta/2}) */
        u[0] = c;  u[1] = -s;
        u[2 * 3] = c;  u[2 * 3 + 1] = s;
        break;
    case K_CZ:
        u[2 * (3 * 4 + 3)] = -1.0;
        break;
    case K_GIVENS: {
        int a = 1, b = 2;            /* |a=1,b=0> -> j=1, |a=0,b=1> -> j=2 */
        u[2 * (a * 4 + a)] = c;  u[2 * (a * 4 + b)] = -s;
        u[2 * (b * 4 + a)] = s;  u[2 * (b * 4 + b)] = c;
        break;
    }
    case K_DEXC: {
        int a = 3, b = 12;           /* q0,q1 set -> 3 ; q2,q3 set -> 12 */
        u[2 * (a * 16 + a)] = c;  u[2 * (a * 16 + b)] = -s;
        u[2 * (b * 16 + a)] = s;  u[2 * (b * 16 + b)] = c;
        break;
    }
    default:
        if (!mat) return -1;
        memcpy(u, mat, sizeof(double) * 2 * dim * dim);
        break;
    }
    if (inverse) {
        /* U^dagger: conjugate transpose */
        double *t = (double *)malloc(sizeof(double) * 2 * dim * dim);
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j) {
                t[2 * (i * dim + j)] = u[2 * (j * dim + i)];
                t[2 * (i * dim + j) + 1] = -u[2 * (j * dim + i) + 1];
            }
        memcpy(u, t, sizeof(double) * 2 * dim * dim);
        free(t);
    }
    return dim;
}

/* Apply a dense dim x dim matrix on the given target qubits. */
static void apply_dense(double *psi, int n, const int *tq, int nq, const double *u) {
    int dim = 1 << nq;
    uint64_t tmask = 0;
    for (int t = 0; t < nq; ++t) tmask |= (uint64_t)1 << tq[t];
    uint64_t N = (uint64_t)1 << n;
    uint64_t nbase = N >> nq;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)nbase; ++r) {
        /* r enumerates the indices with every target bit clear */
        uint64_t base = 0, rem = (uint64_t)r;
        for (int bit = 0; bit < n; ++bit) {
            if (tmask & ((uint64_t)1 << bit)) continue;
            base |= (rem & 1) << bit;
            rem >>= 1;
        }
        double vr[16], vi[16];
        uint64_t idx[16];
        for (int j = 0; j < dim; ++j) {
            uint64_t b = base;
            for (int t = 0; t < nq; ++t)
                if (j & (1 << t)) b |= (uint64_t)1 << tq[t];
            idx[j] = b;
            vr[j] = psi[2 * b];
            vi[j] = psi[2 * b + 1];
        }
        for (int i = 0; i < dim; ++i) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < dim; ++j) {
                double ur = u[2 * (i * dim + j)], ui = u[2 * (i * dim + j) + 1];
                sr += ur * vr[j] - ui * vi[j];
                si += ur * vi[j] + ui * vr[j];
            }
            psi[2 * idx[i]] = sr;
            psi[2 * idx[i] + 1] = si;
        }
    }
}

/*
 * Apply gates 0..m-1 in order (inverse != 0: apply U_{m-1}^dagger first, down
 * to U_0^dagger, i.e. the inverse circuit).  Returns 0 or -1 on bad input.
 */
int osim_apply(double *psi, int n, int m, const int32_t *kinds, const int32_t *qubits,
               const int32_t *param, const int32_t *mat, const double *params,
               const double *mats, int inverse) {
    double u[2 * 16 * 16];
    for (int s = 0; s < m; ++s) {
        int i = inverse ? (m - 1 - s) : s;
        int nq = gate_nq(kinds[i]);
        if (nq < 0) return -1;
        int tq[4];
        for (int t = 0; t < nq; ++t) {
            tq[t] = qubits[4 * i + t];
            if (tq[t] < 0 || tq[t] >= n) return -1;
        }
        double theta = param[i] >= 0 ? params[param[i]] : 0.0;
        const double *mp = (mat && mat[i] >= 0 && mats) ? mats + 2 * (size_t)mat[i] : NULL;
        if (build_matrix(kinds[i], theta, mp, inverse, u) < 0) return -1;
        apply_dense(psi, n, tq, nq, u);
    }
    return 0;
}

/*
 * <psi|P_t|psi> for each string t (letters[t*n + q] in {0:I,1:X,2:Y,3:Z}).
 * P|b> is built qubit by qubit from Eq. (pauli_matrix):
 *   X|0>=|1>, X|1>=|0>;  Y|0>=i|1>, Y|1>=-i|0>;  Z|0>=|0>, Z|1>=-|1>.
 * Then <psi|P|psi> = sum_b conj(psi[b']) * phase(b) * psi[b], b' = image of b.
 * out[2t] = real part, out[2t+1] = imaginary part.
 */
void osim_expect(const double *psi, int n, int nterms, const uint8_t *letters, double *out) {
    uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nterms; ++t) {
        const uint8_t *L = letters + (size_t)t * n;
        int pos[64], code[64], k = 0;
        for (int q = 0; q < n; ++q)
            if (L[q]) { pos[k] = q; code[k] = L[q]; ++k; }
        double acc_r = 0.0, acc_i = 0.0;
        for (uint64_t b = 0; b < N; ++b) {
            double ph_r = 1.0, ph_i = 0.0;   /* phase picked up by |b> */
            uint64_t img = b;
            for (int j = 0; j < k; ++j) {
                int bit = (int)((b >> pos[j]) & 1);
                double fr, fi;
                if (code[j] == 1) {            /* X */
                    fr = 1.0; fi = 0.0;
                    img ^= (uint64_t)1 << pos[j];
                } else if (code[j] == 2) {     /* Y */
                    fr = 0.0; fi = bit ? -1.0 : 1.0;
                    img ^= (uint64_t)1 << pos[j];
                } else {                       /* Z */
                    fr = bit ? -1.0 : 1.0; fi = 0.0;
                }
                double nr = ph_r * fr - ph_i * fi;
                double ni = ph_r * fi + ph_i * fr;
                ph_r = nr; ph_i = ni;
            }
            /* (P psi)[img] gets phase * psi[b]; pair it with conj(psi[img]) */
            double pr = psi[2 * b], pi = psi[2 * b + 1];
            double vr = ph_r * pr - ph_i * pi, vi = ph_r * pi + ph_i * pr;
            double cr = psi[2 * img], ci = -psi[2 * img + 1];
            acc_r += cr * vr - ci * vi;
            acc_i += cr * vi + ci * vr;
        }
        out[2 * t] = acc_r;
        out[2 * t + 1] = acc_i;
    }
}

/* H|psi> as a full vector (used only to pin the library's lambda = H psi):
 * out = sum_t coeff_t P_t psi, built letter by letter as in osim_expect. */
void osim_apply_hamiltonian(const double *psi, int n, int nterms, const uint8_t *letters,
                            const double *coeffs, double *out) {
    uint64_t N = (uint64_t)1 << n;
    memset(out, 0, sizeof(double) * 2 * N);
    for (int t = 0; t < nterms; ++t) {
        const uint8_t *L = letters + (size_t)t * n;
        int pos[64], code[64], k = 0;
        for (int q = 0; q < n; ++q)
            if (L[q]) { pos[k] = q; code[k] = L[q]; ++k; }
        double a = coeffs[t];
#pragma omp parallel for schedule(static)
        for (int64_t bb = 0; bb < (int64_t)N; ++bb) {
            /* out[img] += a * phase(b) * psi[b]; iterate over img instead so
             * that each thread owns its output element: img -> b is the same
             * flip, and the phase is evaluated on b. */
            uint64_t img = (uint64_t)bb, b = img;
            for (int j = 0; j < k; ++j)
                if (code[j] == 1 || code[j] == 2) b ^= (uint64_t)1 << pos[j];
            double ph_r = 1.0, ph_i = 0.0;
            for (int j = 0; j < k; ++j) {
                int bit = (int)((b >> pos[j]) & 1);
                double fr, fi;
                if (code[j] == 1) { fr = 1.0; fi = 0.0; }
                else if (code[j] == 2) { fr = 0.0; fi = bit ? -1.0 : 1.0; }
                else { fr = bit ? -1.0 : 1.0; fi = 0.0; }
                double nr = ph_r * fr - ph_i * fi;
                double ni = ph_r * fi + ph_i * fr;
                ph_r = nr; ph_i = ni;
            }
            double pr = psi[2 * b], pi = psi[2 * b + 1];
            out[2 * img] += a * (ph_r * pr - ph_i * pi);
            out[2 * img + 1] += a * (ph_r * pi + ph_i * pr);
        }
    }
}

/* Gate matrix export (for the tests that pin the conventions above). */
int osim_gate_matrix(int kind, double theta, const double *mat, int inverse, double *u) {
    return build_matrix(kind, theta, mat, inverse, u);
}
