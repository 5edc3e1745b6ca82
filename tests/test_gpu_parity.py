"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded inputs.  Tolerances: complex128 amplitudes 1e-12 max-abs;
complex64 amplitudes 2e-5 max-abs (FP32 gate math over a few hundred gates);
expectations, energies and gradients within 1e-4 * sum|a_t| (the stated
bound for FP32 state with FP64 accumulation)."""
import math

import numpy as np
import pytest

import oracle
from oracle import grad as ograd
from oracle import planner as P
from paper_2410_04252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
sv = pytest.importorskip("paper_2410_04252_gb300.sv")

AMP_TOL = {sv.C64: 2e-5, sv.C128: 1e-12}


def l1(h):
    return float(np.abs(h.coeffs).sum())


def oracle_state(circ, params, init):
    return oracle.apply_circuit(oracle.basis_state(circ.n, init), circ, params)


def mixed_circuit(n, m, seed, with_mats=True):
    kinds = (W.RY, W.RZ, W.CZ, W.GIVENS, W.DEXC) + ((W.MAT1, W.MAT2, W.MAT4) if with_mats else ())
    c = W.random_circuit(n, m, seed, kinds)
    # matrices for MAT gates
    offs, mats = 0, []
    for i in range(c.m):
        k = int(c.kinds[i])
        if k in (W.MAT1, W.MAT2, W.MAT4):
            dim = 1 << W.GATE_NQ[k]
            mats.append(W.random_unitary_mats(1, dim, seed * 1000 + i))
            c.mat[i] = offs
            offs += dim * dim
    c.mats = np.concatenate(mats) if mats else np.zeros(0)
    return c


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("sched", [sv.LAZY, sv.EAGER])
@pytest.mark.parametrize("n,g", [(6, 2), (9, 3), (12, 2), (14, 4), (15, 0)])
def test_qsu_random_circuits(dtype, sched, n, g):
    c = mixed_circuit(n, 60, 17 + n + g)
    params = W.uniform_params(c.nparams, 3 + n, -math.pi, math.pi)
    s = sv.StateVector(n, g, dtype)
    s.reset(5)
    s.apply_circuit(c, params, sched)
    # the layout the library ends in is the oracle planner's
    T = [c.targets(i) for i in range(c.m)]
    plan = P.flat_tiling(n, T, n - g) if sched == sv.LAZY else P.adhoc_schedule(n, T, n - g)
    if plan.perms:
        assert list(s.permutation()) == plan.perms[-1]
    got = s.get_state(logical=True)
    ref = oracle_state(c, params, 5)
    assert np.max(np.abs(got - ref)) < AMP_TOL[dtype]


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
def test_qsu_paper_ansatze(dtype):
    for ansatz, n, g, layers in [("hea", 16, 4, 4), ("fabric", 18, 4, 6), ("hea", 20, 6, 2)]:
        c = W.hea_circuit(n, layers) if ansatz == "hea" else W.fabric_circuit(n, layers)
        params = W.uniform_params(c.nparams, 7, -math.pi, math.pi)
        init = 0 if ansatz == "hea" else W.half_filled_index(n)
        ref = oracle_state(c, params, init)
        for sched in (sv.LAZY, sv.EAGER):
            s = sv.StateVector(n, g, dtype)
            s.reset(init)
            s.apply_circuit(c, params, sched)
            got = s.get_state(logical=True)
            assert np.max(np.abs(got - ref)) < AMP_TOL[dtype] * (4 if dtype == sv.C64 else 1)


@pytest.mark.parametrize("tile_bits,low_bits", [(9, 3), (11, 5), (13, 4), (13, 1)])
def test_qsu_tile_options(tile_bits, low_bits):
    n, g = 16, 3
    c = mixed_circuit(n, 80, 5)
    params = W.uniform_params(c.nparams, 8, -3, 3)
    o = sv.default_options(sv.C64)
    o.tile_bits, o.low_bits = tile_bits, low_bits
    s = sv.StateVector(n, g, sv.C64, options=o)
    s.reset(3)
    s.apply_circuit(c, params, sv.LAZY)
    assert np.max(np.abs(s.get_state() - oracle_state(c, params, 3))) < 2e-5


def test_qsu_edge_cases():
    # empty circuit; n = 4 with g = 0; a circuit using every qubit of n = 5
    s = sv.StateVector(8, 2, sv.C128)
    s.reset(77)
    s.apply_circuit(W._circuit(8, [], 0), np.zeros(0), sv.LAZY)
    ref = np.zeros(256, complex)
    ref[77] = 1
    assert np.max(np.abs(s.get_state() - ref)) == 0
    c = mixed_circuit(4, 30, 2)
    p = W.uniform_params(c.nparams, 2, -1, 1)
    s = sv.StateVector(4, 0, sv.C128)
    s.reset(0)
    s.apply_circuit(c, p, sv.LAZY)
    assert np.max(np.abs(s.get_state() - oracle_state(c, p, 0))) < 1e-12
    # invalid inputs raise, nothing runs
    with pytest.raises(sv.SvError):
        s.apply_circuit(W._circuit(4, [(W.RY, (9,), 0, -1)], 1), np.zeros(1), sv.LAZY)
    with pytest.raises(sv.SvError):
        s.apply_circuit(W._circuit(4, [(W.RY, (1,), 0, -1)], 1), np.array([np.nan]), sv.LAZY)


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("sched", [sv.LAZY, sv.EAGER])
@pytest.mark.parametrize("kind,n,g", [("random", 10, 2), ("random", 14, 3), ("jw", 12, 3), ("jw", 16, 4),
                                        ("random", 17, 3), ("jw", 17, 3)])
def test_evc(dtype, sched, kind, n, g):
    h = W.random_hamiltonian(n, 64, 31 + n) if kind == "random" else W.jw_hamiltonian(n, 256, 33 + n)
    c = W.hea_circuit(n, 2)
    params = W.uniform_params(c.nparams, 4, 0, 2 * math.pi)
    psi = oracle_state(c, params, 0)
    ref_terms = oracle.expect_terms(psi, h).real
    ref_e = float(np.dot(h.coeffs, ref_terms))
    s = sv.StateVector(n, g, dtype)
    s.reset(0)
    s.apply_circuit(c, params, sv.LAZY)
    e, pt = s.expect(h, sched)
    tol = 1e-12 if dtype == sv.C128 else 1e-4 * l1(h)
    assert abs(e - ref_e) < tol
    assert np.max(np.abs(pt - ref_terms)) < (1e-12 if dtype == sv.C128 else 2e-5)


def test_evc_special_strings_and_keep_layout():
    n, g = 12, 3
    L = np.zeros((6, n), np.uint8)
    L[1, :] = 3                       # Z on every qubit (Z on all global qubits too)
    L[2, 0] = 1; L[2, n - 1] = 2      # X on a local and Y on a global qubit
    L[3, :n - g + 1] = 1              # X on more qubits than are local: no mapping fits
    L[4, 5] = 2
    L[5, 2] = 1; L[5, 3] = 1; L[5, 11] = 3
    h = W.Hamiltonian(n, L, np.array([0.5, -1.0, 0.3, 0.7, 1.1, -0.2]))   # row 0: identity
    c = W.hea_circuit(n, 3)
    params = W.uniform_params(c.nparams, 9, 0, 2 * math.pi)
    psi = oracle_state(c, params, 0)
    ref = oracle.expect_terms(psi, h).real
    assert abs(ref[0] - 1) < 1e-12
    s = sv.StateVector(n, g, sv.C128)
    s.reset(0)
    s.apply_circuit(c, params, sv.LAZY)
    before = list(s.permutation())
    e, pt = s.expect(h, sv.LAZY, keep_layout=True)
    assert list(s.permutation()) == before
    np.testing.assert_allclose(pt, ref, atol=1e-12)
    assert abs(e - np.dot(h.coeffs, ref)) < 1e-12
    np.testing.assert_allclose(s.get_state(), psi, atol=1e-12)


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("kind", ["random", "jw"])
def test_apply_hamiltonian(dtype, kind):
    n, g = 13, 3
    h = W.random_hamiltonian(n, 100, 5) if kind == "random" else W.jw_hamiltonian(n, 200, 6)
    c = W.hea_circuit(n, 2)
    params = W.uniform_params(c.nparams, 4, 0, 2 * math.pi)
    psi = oracle_state(c, params, 0)
    ref = oracle.apply_hamiltonian(psi, h)
    s = sv.StateVector(n, g, dtype)
    s.set_state(psi)
    e, lam = s.apply_hamiltonian(h)
    lam = lam.cpu().numpy()
    tol = 1e-11 if dtype == sv.C128 else 1e-4 * l1(h)
    assert np.max(np.abs(lam - ref)) < tol
    assert abs(e - oracle.energy(psi, h)) < tol


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("sched", [sv.LAZY, sv.EAGER])
def test_adjoint_gradient_hea(dtype, sched):
    n, g = 10, 3
    c = W.hea_circuit(n, 3)
    params = W.uniform_params(c.nparams, 12, 0, 2 * math.pi)
    h = W.random_hamiltonian(n, 48, 13)
    ps = ograd.parameter_shift(c, params, h)
    e_ref = ograd.objective(c, params, h)
    s = sv.StateVector(n, g, dtype)
    s.reset(0)
    e, gr = s.grad(c, params, h, sched)
    tol = 1e-10 if dtype == sv.C128 else 1e-4 * l1(h)
    assert abs(e - e_ref) < tol
    assert np.max(np.abs(gr - ps)) < tol
    # the sweep returns the state to |psi0>
    back = s.get_state()
    assert abs(back[0] - 1) < (1e-10 if dtype == sv.C128 else 1e-4)


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
def test_adjoint_gradient_fabric_and_mixed(dtype):
    n, g = 10, 2
    c = W.fabric_circuit(n, 4)
    params = W.uniform_params(c.nparams, 14, -math.pi, math.pi)
    h = W.jw_hamiltonian(n, 80, 15)
    init = W.half_filled_index(n)
    fd = ograd.finite_difference(c, params, h, init)
    s = sv.StateVector(n, g, dtype)
    s.reset(init)
    e, gr = s.grad(c, params, h, sv.LAZY)
    tol = 1e-7 if dtype == sv.C128 else 1e-4 * l1(h)
    assert abs(e - ograd.objective(c, params, h, init)) < tol
    assert np.max(np.abs(gr - fd)) < tol
    # random circuit with fixed matrices mixed in (no parameters on them)
    c2 = mixed_circuit(9, 50, 3)
    p2 = W.uniform_params(c2.nparams, 16, -2, 2)
    h2 = W.random_hamiltonian(9, 30, 17)
    fd2 = ograd.finite_difference(c2, p2, h2, 6)
    s2 = sv.StateVector(9, 2, dtype)
    s2.reset(6)
    e2, g2 = s2.grad(c2, p2, h2, sv.EAGER)
    assert np.max(np.abs(g2 - fd2)) < (1e-7 if dtype == sv.C128 else 1e-4 * l1(h2))


def test_vqe_step_matches_parts_and_is_deterministic():
    n, g = 12, 3
    c = W.hea_circuit(n, 3)
    params = W.uniform_params(c.nparams, 21, 0, 2 * math.pi)
    h = W.random_hamiltonian(n, 64, 22)
    s = sv.StateVector(n, g, sv.C64)
    e1, g1, pt1 = s.vqe_step(0, c, params, h, sv.LAZY, per_term=True)
    e2, g2, pt2 = s.vqe_step(0, c, params, h, sv.LAZY, per_term=True)
    assert e1 == e2 and np.array_equal(g1, g2) and np.array_equal(pt1, pt2)    # bitwise
    ps = ograd.parameter_shift(c, params, h)
    assert np.max(np.abs(g1 - ps)) < 1e-4 * l1(h)
    assert abs(e1 - ograd.objective(c, params, h)) < 1e-4 * l1(h)
    e3, g3, _ = s.vqe_step(0, c, params, h, sv.EAGER)
    assert abs(e3 - e1) < 1e-4 * l1(h)
    assert np.max(np.abs(g3 - g1)) < 1e-4 * l1(h)


@pytest.mark.parametrize("every", [1, 2])
def test_adjoint_with_forward_checkpoints(every):
    """Re-anchoring psi from forward checkpoints gives the same gradient and
    leaves the state at |psi0>; the checkpoints are dropped afterwards."""
    n, g = 13, 3
    c = W.hea_circuit(n, 4)
    params = W.uniform_params(c.nparams, 31, 0, 2 * math.pi)
    h = W.random_hamiltonian(n, 40, 32)
    o = sv.default_options(sv.C64)
    o.tile_bits, o.low_bits = 9, 3            # several passes so checkpoints are taken
    s0 = sv.StateVector(n, g, sv.C64, options=o)
    s0.reset(0)
    e0, g0 = s0.grad(c, params, h, sv.LAZY)
    o.checkpoint_every = every
    s1 = sv.StateVector(n, g, sv.C64, options=o)
    s1.reset(0)
    e1, g1 = s1.grad(c, params, h, sv.LAZY)
    st = s1.last_stats
    assert st.kernels[sv.K_PERM] > 0          # checkpoint copies were made and used
    assert abs(e1 - e0) < 1e-4 * float(np.abs(h.coeffs).sum())
    assert np.max(np.abs(g1 - g0)) < 1e-4 * float(np.abs(h.coeffs).sum())
    ps = ograd.parameter_shift(c, params, h)
    assert np.max(np.abs(g1 - ps)) < 1e-4 * float(np.abs(h.coeffs).sum())
    assert abs(s1.get_state()[0] - 1) < 1e-4
    # vqe_step (forward by sv_apply_circuit, gradient with SV_FORWARD_DONE) uses them too
    e2, g2, _ = s1.vqe_step(0, c, params, h, sv.LAZY)
    assert np.max(np.abs(g2 - ps)) < 1e-4 * float(np.abs(h.coeffs).sum())


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
def test_direct_schedule(dtype):
    """DIRECT (no virtual-chunk constraint, no QR) gives the oracle's state,
    expectations and gradient."""
    n, g = 14, 4
    c = mixed_circuit(n, 80, 123, with_mats=False)
    p = W.uniform_params(c.nparams, 124, -math.pi, math.pi)
    s = sv.StateVector(n, g, dtype)
    s.reset(3)
    st = s.apply_circuit(c, p, sv.DIRECT)
    assert st.qsu_qrs == 0
    ref = oracle_state(c, p, 3)
    assert np.max(np.abs(s.get_state() - ref)) < AMP_TOL[dtype]
    ham = W.jw_hamiltonian(n, 200, 125)
    e, pt = s.expect(ham, sv.DIRECT)
    assert s.last_stats.evc_qrs == 0
    tol = 1e-4 * l1(ham) if dtype == sv.C64 else 1e-10 * l1(ham)
    assert abs(e - oracle.energy(ref, ham)) < tol
    h2 = W.random_hamiltonian(n, 64, 126)
    e2, gr, _ = s.vqe_step(0, c, p, h2, sv.DIRECT)
    tol2 = 1e-4 * l1(h2) if dtype == sv.C64 else 1e-7
    assert abs(e2 - ograd.objective(c, p, h2)) < tol2
    # Givens / double-excitation parameters: central differences
    assert np.max(np.abs(gr - ograd.finite_difference(c, p, h2))) < tol2


@pytest.mark.parametrize("ni", [0, 1, 3])
def test_hierarchical_schedule(ni):
    """QSU under hierarchical tiling (Alg. 4/5) gives the oracle's state; its
    layout is the oracle planner's; the gradient under it is the oracle's."""
    n, g = 13, 3
    c = W.fabric_circuit(n, 6)
    p = W.uniform_params(c.nparams, 131, -math.pi, math.pi)
    init = W.half_filled_index(n)
    o = sv.default_options(sv.C64)
    o.intra_bits = ni
    s = sv.StateVector(n, g, sv.C64, options=o)
    s.reset(init)
    s.apply_circuit(c, p, sv.HIER)
    T = [c.targets(i) for i in range(c.m)]
    plan = P.hierarchical_tiling(n, T, n - g, ni)
    assert list(s.permutation()) == plan.perms[-1]
    ref = oracle_state(c, p, init)
    assert np.max(np.abs(s.get_state() - ref)) < AMP_TOL[sv.C64]
    h = W.jw_hamiltonian(n, 90, 132)
    s.reset(init)
    e, gr = s.grad(c, p, h, sv.HIER)
    assert abs(e - ograd.objective(c, p, h, init)) < 1e-4 * l1(h)
    assert np.max(np.abs(gr - ograd.finite_difference(c, p, h, init))) < 1e-4 * l1(h)


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("fuse_max", [0, 20])
def test_register_passes_full_tiles(dtype, fuse_max):
    """HEA with the largest staged tiles (k = 13 for complex64, 12 for
    complex128: 16 / 8 amplitudes per thread in the register phases, with
    diagonal blocks of RZ / CZ runs): state, energy and gradient against the
    oracle; fuse_max = 20 cuts the passes so that blocks start and end
    inside phases differently."""
    n, g = 16, 2
    c = W.hea_circuit(n, 3)
    p = W.uniform_params(c.nparams, 141, 0, 2 * math.pi)
    o = sv.default_options(dtype)
    o.fuse_max = fuse_max
    s = sv.StateVector(n, g, dtype, options=o)
    s.reset(0)
    s.apply_circuit(c, p, sv.LAZY)
    ref = oracle_state(c, p, 0)
    assert np.max(np.abs(s.get_state() - ref)) < AMP_TOL[dtype]
    h = W.random_hamiltonian(n, 40, 142)
    e, gr, _ = s.vqe_step(0, c, p, h, sv.LAZY)
    tol = 1e-4 * l1(h) if dtype == sv.C64 else 1e-10 * l1(h)
    assert abs(e - ograd.objective(c, p, h)) < tol
    assert np.max(np.abs(gr - ograd.parameter_shift(c, p, h))) < tol


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("n,g,kinds", [(14, 4, "rzcz"), (16, 3, "rzcz"), (13, 3, "givens")])
def test_diagonal_exemption_schedule(dtype, n, g, kinds):
    """LAZY_DIAG: diagonal gates on global qubits applied as per-tile phases /
    signs (register-phased passes for RY/RZ/CZ circuits, plain passes when a
    Givens gate is in the pass): state, energy and gradient = oracle."""
    ks = (W.RY, W.RZ, W.CZ) if kinds == "rzcz" else (W.RY, W.RZ, W.CZ, W.GIVENS)
    c = W.random_circuit(n, 160, 300 + n + g, ks)
    p = W.uniform_params(c.nparams, 301 + n, -math.pi, math.pi)
    s = sv.StateVector(n, g, dtype)
    s.reset(5)
    st = s.apply_circuit(c, p, sv.LAZY_DIAG)
    lz = sv.plan_qsu(n, g, c, sv.LAZY)
    assert st.qsu_qrs <= sum(1 for t in lz["tiles"] if t["pairs"])
    ref = oracle_state(c, p, 5)
    assert np.max(np.abs(s.get_state() - ref)) < AMP_TOL[dtype]
    h = W.random_hamiltonian(n, 48, 302 + n)
    e, gr, _ = s.vqe_step(5, c, p, h, sv.LAZY_DIAG)
    tol = 1e-4 * l1(h) if dtype == sv.C64 else 1e-7
    assert abs(e - ograd.objective(c, p, h, 5)) < tol
    assert np.max(np.abs(gr - ograd.finite_difference(c, p, h, 5))) < tol


@pytest.mark.parametrize("sched", [sv.LAZY, sv.DIRECT])
def test_evc_large_groups(sched):
    """Groups of many strings sharing one x-mask (pure-Z terms, and X/Y masks
    with many Z variants of both nY parities) on 8192-amplitude cosets: the
    per-group transform path (>= 16 strings, with and without X) and the
    per-string fold path (fewer) of the EVC pass, per term against the
    oracle."""
    n, g = 17, 3
    rng = np.random.default_rng(4242)
    rows = []
    for _ in range(70):                                   # pure Z, any weight, global qubits included
        r = np.zeros(n, np.uint8)
        r[rng.random(n) < 0.3] = 3
        rows.append(r)
    for size, nvar in ((2, 14), (3, 24), (4, 14)):       # three x-masks with 14 or 24 Z/Y variants
        xs = rng.choice(n - g, size, replace=False)
        for _ in range(nvar):
            r = np.zeros(n, np.uint8)
            r[rng.random(n) < 0.4] = 3
            r[xs] = rng.choice([1, 2], size)
            rows.append(r)
    for _ in range(20):                                   # scattered strings (single-string groups)
        rows.append(rng.integers(0, 4, n).astype(np.uint8))
    L = np.unique(np.array(rows), axis=0)
    h = W.Hamiltonian(n, L, rng.normal(size=len(L)))
    c = W.hea_circuit(n, 2)
    params = W.uniform_params(c.nparams, 44, 0, 2 * math.pi)
    psi = oracle_state(c, params, 0)
    ref_terms = oracle.expect_terms(psi, h).real
    s = sv.StateVector(n, g, sv.C64)
    s.reset(0)
    s.apply_circuit(c, params, sv.LAZY)
    e, pt = s.expect(h, sched)
    assert np.max(np.abs(pt - ref_terms)) < 2e-5
    assert abs(e - float(np.dot(h.coeffs, ref_terms))) < 1e-4 * l1(h)


@pytest.mark.parametrize("kind", ["random", "jw"])
def test_adjoint_gradient_fast_coset_paths(kind):
    """14 local qubits give 8192-amplitude cosets under the lazy schedule, the
    shape of the n = 32 workload: the table-driven lambda = H psi pass (random
    strings) and its general fallback (JW passes with many strings) inside
    the gradient, against the parameter-shift rule."""
    n, g = 17, 3
    c = W.hea_circuit(n, 1)
    params = W.uniform_params(c.nparams, 71, 0, 2 * math.pi)
    h = W.random_hamiltonian(n, 48, 72) if kind == "random" else W.jw_hamiltonian(n, 120, 73)
    s = sv.StateVector(n, g, sv.C64)
    s.reset(0)
    e, gr = s.grad(c, params, h, sv.LAZY)
    tol = 1e-4 * l1(h)
    assert abs(e - ograd.objective(c, params, h)) < tol
    assert np.max(np.abs(gr - ograd.parameter_shift(c, params, h))) < tol
