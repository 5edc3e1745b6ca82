"""Pins for the oracle simulator (oracle/svsim.c) against things other than
itself: generators exponentiated with scipy, dense Pauli matrices built by
Kronecker products, closed forms and invariants."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2410_04252_gb300 import workloads as W

I2 = np.eye(2, dtype=complex)
X2 = np.array([[0, 1], [1, 0]], dtype=complex)
Y2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z2 = np.array([[1, 0], [0, -1]], dtype=complex)
LETTER = {0: I2, 1: X2, 2: Y2, 3: Z2}


def op_on(n, q, m2):
    """Full-space operator acting as m2 on qubit q (index bit q), built by
    Kronecker products with the most significant qubit first."""
    out = np.array([[1.0 + 0j]])
    for k in range(n - 1, -1, -1):
        out = np.kron(out, m2 if k == q else I2)
    return out


def raise_op(n, q):   # |1><0| on qubit q
    return op_on(n, q, (X2 - 1j * Y2) / 2)


def lower_op(n, q):   # |0><1| on qubit q
    return op_on(n, q, (X2 + 1j * Y2) / 2)


def generator(n, kind, qs):
    if kind == W.RY:
        return op_on(n, qs[0], Y2)
    if kind == W.RZ:
        return op_on(n, qs[0], Z2)
    if kind == W.GIVENS:
        a, b = qs
        # i (R_b L_a - R_a L_b): |a=1,b=0> -> i |a=0,b=1>
        return 1j * (raise_op(n, b) @ lower_op(n, a) - raise_op(n, a) @ lower_op(n, b))
    if kind == W.DEXC:
        q0, q1, q2, q3 = qs
        fwd = raise_op(n, q2) @ raise_op(n, q3) @ lower_op(n, q0) @ lower_op(n, q1)
        bwd = raise_op(n, q0) @ raise_op(n, q1) @ lower_op(n, q2) @ lower_op(n, q3)
        return 1j * (fwd - bwd)
    raise ValueError


def oracle_full_matrix(circ, params, inverse=False):
    n = circ.n
    cols = []
    for b in range(1 << n):
        cols.append(oracle.apply_circuit(oracle.basis_state(n, b), circ, params, inverse))
    return np.stack(cols, axis=1)


def single_gate(n, kind, qs, theta=0.0, mat=None):
    p = 0 if kind in (W.RY, W.RZ, W.GIVENS, W.DEXC) else -1
    mi = 0 if mat is not None else -1
    c = W._circuit(n, [(kind, tuple(qs), p, mi)], 1 if p == 0 else 0, mats=mat)
    return c, np.array([theta])


@pytest.mark.parametrize("kind,qs", [(W.RY, (2,)), (W.RZ, (0,)), (W.GIVENS, (3, 1)),
                                     (W.GIVENS, (0, 4)), (W.DEXC, (0, 1, 2, 3)),
                                     (W.DEXC, (4, 1, 0, 3))])
def test_gates_are_exp_of_generator(kind, qs):
    n = 5
    for theta in (0.3, -1.7, 2.9):
        c, p = single_gate(n, kind, qs, theta)
        U = oracle_full_matrix(c, p)
        ref = expm(-0.5j * theta * generator(n, kind, qs))
        np.testing.assert_allclose(U, ref, atol=1e-13)
        Uinv = oracle_full_matrix(c, p, inverse=True)
        np.testing.assert_allclose(Uinv, ref.conj().T, atol=1e-13)


def test_cz_is_controlled_z():
    n = 4
    c, p = single_gate(n, W.CZ, (3, 1))
    U = oracle_full_matrix(c, p)
    # CZ = (I + Z_a + Z_b - Z_a Z_b) / 2
    za, zb = op_on(n, 3, Z2), op_on(n, 1, Z2)
    ref = (np.eye(1 << n) + za + zb - za @ zb) / 2
    np.testing.assert_allclose(U, ref, atol=1e-15)


@pytest.mark.parametrize("kind,dim,qs", [(W.MAT1, 2, (3,)), (W.MAT2, 4, (4, 0)),
                                         (W.MAT4, 16, (1, 5, 0, 3))])
def test_dense_matrix_gate_embedding(kind, dim, qs):
    """A caller matrix acts on its targets with target t <-> matrix index bit t."""
    n = 6
    mats = W.random_unitary_mats(1, dim, seed=11)
    c, p = single_gate(n, kind, qs, mat=mats)
    U = oracle_full_matrix(c, p)
    M = (mats[0::2] + 1j * mats[1::2]).reshape(dim, dim)
    ref = np.zeros((1 << n, 1 << n), complex)
    for b in range(1 << n):
        j = sum(((b >> q) & 1) << t for t, q in enumerate(qs))
        rest = b & ~sum(1 << q for q in qs)
        for i in range(dim):
            bb = rest | sum(((i >> t) & 1) << q for t, q in enumerate(qs))
            ref[bb, b] = M[i, j]
    np.testing.assert_allclose(U, ref, atol=1e-14)


def pauli_dense(letters):
    n = len(letters)
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, LETTER[int(letters[q])])
    return out


def rand_state(n, seed):
    rng = W.SplitMix64(seed)
    v = np.array([complex(rng.normal(), rng.normal()) for _ in range(1 << n)])
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [1, 3, 6, 8])
def test_expect_matches_dense_pauli_matrices(n):
    ham = W.random_hamiltonian(n, 24, seed=5 + n)
    psi = rand_state(n, 100 + n)
    got = oracle.expect_terms(psi, ham)
    for t in range(ham.nterms):
        P = pauli_dense(ham.letters[t])
        ref = np.vdot(psi, P @ psi)
        assert abs(got[t] - ref) < 1e-12
        assert abs(got[t].imag) < 1e-12      # Hermitian P
    E = oracle.energy(psi, ham)
    Hd = sum(a * pauli_dense(ham.letters[t]) for t, a in enumerate(ham.coeffs))
    assert abs(E - np.vdot(psi, Hd @ psi).real) < 1e-11
    Hpsi = oracle.apply_hamiltonian(psi, ham)
    np.testing.assert_allclose(Hpsi, Hd @ psi, atol=1e-12)


def test_ry_closed_forms():
    for theta in (0.0, 0.4, 1.3, -2.2, math.pi):
        c, p = single_gate(1, W.RY, (0,), theta)
        psi = oracle.apply_circuit(oracle.basis_state(1, 0), c, p)
        h = W.Hamiltonian(1, np.array([[3], [1], [2]], np.uint8), np.ones(3))
        e = oracle.expect_terms(psi, h).real
        assert abs(e[0] - math.cos(theta)) < 1e-14
        assert abs(e[1] - math.sin(theta)) < 1e-14
        assert abs(e[2]) < 1e-14


def test_ghz_parities():
    n = 7
    psi = np.zeros(1 << n, complex)
    psi[0] = psi[-1] = 1 / math.sqrt(2)
    L = []
    L.append([3, 3] + [0] * (n - 2))           # Z0 Z1 -> 1
    L.append([0] * 3 + [3] + [0] * (n - 4))     # Z3 -> 0
    L.append([1] * n)                           # X^n -> 1
    L.append([2, 2] + [1] * (n - 2))            # Y Y X..X -> -1
    L.append([2] * 4 + [1] * (n - 4))           # Y^4 X.. -> +1 (i^4 = 1)
    h = W.Hamiltonian(n, np.array(L, np.uint8), np.ones(len(L)))
    e = oracle.expect_terms(psi, h)
    np.testing.assert_allclose(e, [1, 0, 1, -1, 1], atol=1e-14)


def test_product_state_factorises():
    n = 5
    thetas = [0.3, 1.1, -0.7, 2.5, 0.9]
    phis = [0.2, -1.4, 0.5, 3.0, -2.2]
    gates = []
    for q in range(n):
        gates.append((W.RY, (q,), 2 * q, -1))
        gates.append((W.RZ, (q,), 2 * q + 1, -1))
    c = W._circuit(n, gates, 2 * n)
    params = np.array([v for q in range(n) for v in (thetas[q], phis[q])])
    psi = oracle.apply_circuit(oracle.basis_state(n, 0), c, params)
    # single-qubit Bloch vectors: <X>=sin t cos p, <Y>=sin t sin p, <Z>=cos t
    bloch = {1: [math.sin(t) * math.cos(p) for t, p in zip(thetas, phis)],
             2: [math.sin(t) * math.sin(p) for t, p in zip(thetas, phis)],
             3: [math.cos(t) for t in thetas]}
    ham = W.random_hamiltonian(n, 40, seed=77)
    e = oracle.expect_terms(psi, ham)
    for t in range(ham.nterms):
        ref = 1.0
        for q in range(n):
            if ham.letters[t, q]:
                ref *= bloch[int(ham.letters[t, q])][q]
        assert abs(e[t] - ref) < 1e-13


def test_norm_inverse_and_particle_number():
    n = 10
    circ = W.fabric_circuit(n, 4)
    params = W.uniform_params(circ.nparams, 9, -math.pi, math.pi)
    init = W.half_filled_index(n)
    psi = oracle.apply_circuit(oracle.basis_state(n, init), circ, params)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    weights = np.array([bin(b).count("1") for b in range(1 << n)])
    assert np.all(psi[weights != n // 2] == 0)
    assert np.sum(np.abs(psi[weights == n // 2]) ** 2) > 0.999999
    back = oracle.apply_circuit(psi, circ, params, inverse=True)
    assert abs(back[init] - 1) < 1e-12
    circ2 = W.hea_circuit(n, 3)
    p2 = W.uniform_params(circ2.nparams, 3, 0, 2 * math.pi)
    psi2 = oracle.apply_circuit(oracle.basis_state(n, 0), circ2, p2)
    assert abs(np.linalg.norm(psi2) - 1) < 1e-13


def test_any_c1_schedule_gives_same_state():
    """Eq. update_sv_reorder: any order that keeps each qubit's gate sequence
    gives the same final state (brute force over random topological orders)."""
    n = 6
    circ = W.random_circuit(n, 40, seed=21)
    params = W.uniform_params(circ.nparams, 22, -3, 3)
    ref = oracle.apply_circuit(oracle.basis_state(n, 5), circ, params)
    rng = W.SplitMix64(23)
    T = [circ.targets(i) for i in range(circ.m)]
    for _ in range(5):
        done, order = set(), []
        while len(order) < circ.m:
            ready = [i for i in range(circ.m) if i not in done and
                     all(j in done for j in range(i) if set(T[j]) & set(T[i]))]
            pick = ready[rng.randint(len(ready))]
            done.add(pick)
            order.append(pick)
        sub = W.Circuit(n, circ.kinds[order], circ.qubits[order], circ.param[order],
                        circ.mat[order], circ.nparams)
        got = oracle.apply_circuit(oracle.basis_state(n, 5), sub, params)
        np.testing.assert_allclose(got, ref, atol=1e-13)
