"""Full-size correctness at n = 32 (2^32 amplitudes, so every kernel walks
indices above 2^31), where the FP64 oracle cannot run: a product-state
circuit has closed-form expectations and gradients.

The circuit is the 6-layer hardware-efficient ansatz of the n = 32 workload
with its CZ gates removed (RY then RZ on every qubit, 384 parameters), so the
state stays a product of one-qubit states.  For a Pauli string P = (x) sigma_q,
<P> = prod_q <sigma_q> (product states factorise), and the derivative of the
energy by a parameter of qubit q is the derivative of that one factor times
the product of the others.  The one-qubit states, their Bloch components and
their derivatives (dU/dtheta = -i/2 G U for U = exp(-i theta G / 2), G = Y
for RY, Z for RZ) are computed here on the host in FP64 from 2 x 2 matrices.

The last layer's angles are chosen per qubit so that its Bloch vector lies
0.1 rad from a drawn axis; the Hamiltonian's strings mostly carry that axis'
letter, so that the expectations are O(1) instead of vanishingly small, and
carry X/Y letters on the global qubits too.  The whole iteration runs
through sv_vqe_step under the lazy schedule: gate passes, QRs, EVC coset
passes, H|psi> passes and the adjoint sweep."""
import math

import numpy as np
import pytest

from paper_2410_04252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
sv = pytest.importorskip("paper_2410_04252_gb300.sv")

N, G, LAYERS, NTERMS = 32, 6, 6, 1024

_I2 = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)
_SIG = {W.PX: _X, W.PY: _Y, W.PZ: _Z}


def _ry(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=complex)


def _rz(t):
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=complex)


def product_circuit():
    """The ansatz without its CZ gates (same gate order and parameter slots)."""
    full = W.hea_circuit(N, LAYERS)
    keep = np.array([k in (W.RY, W.RZ) for k in full.kinds])
    return W.Circuit(N, full.kinds[keep].copy(), full.qubits[keep].copy(), full.param[keep].copy(),
                     full.mat[keep].copy(), full.nparams)


def _qubit_ops(q, params):
    """(matrix, generator, parameter index) of qubit q's gates in circuit order."""
    ops = []
    for l in range(LAYERS):
        pt, pp = 2 * N * l + q, 2 * N * l + N + q
        ops.append((_ry(params[pt]), _Y, pt))
        ops.append((_rz(params[pp]), _Z, pp))
    return ops


def _bloch(v):
    return np.array([np.vdot(v, s @ v).real for s in (_X, _Y, _Z)])


def choose_params(seed):
    """Random angles for the first five layers; the last layer's RY/RZ angles
    put each qubit 0.1 rad from a drawn signed axis (grid search)."""
    params = W.uniform_params(2 * N * LAYERS, seed, 0.0, 2.0 * math.pi)
    rng = W.SplitMix64(seed + 77)
    axes = np.zeros(N, np.int64)
    grid = np.linspace(0.0, 2.0 * math.pi, 4096, endpoint=False)
    for q in range(N):
        axis = rng.randint(3)
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        axes[q] = axis + 1                                  # letter code X=1, Y=2, Z=3
        tilt, az = 0.1, 2.0 * math.pi * rng.uniform()
        t = np.zeros(3)
        t[axis] = sign * math.cos(tilt)
        t[(axis + 1) % 3] = math.sin(tilt) * math.cos(az)
        t[(axis + 2) % 3] = math.sin(tilt) * math.sin(az)
        v = np.array([1, 0], dtype=complex)
        for mat, _, _ in _qubit_ops(q, params)[:-2]:
            v = mat @ v
        # RY(theta) then RZ(phi): RZ keeps <Z>, so theta fixes <Z>, then phi the azimuth
        zs = np.array([_bloch(_ry(th) @ v)[2] for th in grid])
        th = grid[int(np.argmin(np.abs(zs - t[2])))]
        w = _ry(th) @ v
        al = np.array([_bloch(_rz(ph) @ w) @ t for ph in grid])
        ph = grid[int(np.argmax(al))]
        params[2 * N * (LAYERS - 1) + q] = th
        params[2 * N * (LAYERS - 1) + N + q] = ph
    return params, axes


def make_hamiltonian(axes, seed):
    """Per qubit: I with p = 1/2, the qubit's axis letter with p = 0.45, a
    random other letter with p = 0.05; coefficients N(0, 1)."""
    rng = W.SplitMix64(seed)
    letters = np.zeros((NTERMS, N), np.uint8)
    coeffs = np.zeros(NTERMS, np.float64)
    for t in range(NTERMS):
        for q in range(N):
            u = rng.uniform()
            if u < 0.5:
                letters[t, q] = W.PI
            elif u < 0.95:
                letters[t, q] = axes[q]
            else:
                others = [c for c in (W.PX, W.PY, W.PZ) if c != axes[q]]
                letters[t, q] = others[rng.randint(2)]
        coeffs[t] = rng.normal(1.0)
    return W.Hamiltonian(N, letters, coeffs)


def closed_form(params, ham):
    """Per-term <P_t>, energy and dE/dparams of the product state, FP64."""
    f = np.ones((N, 4))                     # f[q, letter] = <sigma_letter> of qubit q
    df = {}                                 # parameter -> (qubit, d f[q, letter] / d parameter)
    for q in range(N):
        ops = _qubit_ops(q, params)
        v = np.array([1, 0], dtype=complex)
        for mat, _, _ in ops:
            v = mat @ v
        for c, s in _SIG.items():
            f[q, c] = np.vdot(v, s @ v).real
        for i, (_, gen, p) in enumerate(ops):
            dv = np.array([1, 0], dtype=complex)
            for j, (mat, _, _) in enumerate(ops):
                dv = mat @ dv
                if j == i:
                    dv = -0.5j * (gen @ dv)
            d = np.zeros(4)
            for c, s in _SIG.items():
                d[c] = 2.0 * np.vdot(v, s @ dv).real
            df[p] = (q, d)
    L = ham.letters.astype(np.int64)
    fac = f[np.arange(N)[None, :], L]       # [terms, qubits]
    terms = fac.prod(axis=1)
    energy = float(ham.coeffs @ terms)
    grad = np.zeros(len(params))
    for p, (q, d) in df.items():
        others = np.prod(np.delete(fac, q, axis=1), axis=1)
        grad[p] = float(ham.coeffs @ (d[L[:, q]] * others))
    return terms, energy, grad


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
def test_product_state_n32_closed_form(dtype):
    circ = product_circuit()
    params, axes = choose_params(1003)
    ham = make_hamiltonian(axes, 2003)
    terms, energy, grad = closed_form(params, ham)
    assert np.max(np.abs(terms)) > 0.5          # the check is not against values near zero
    l1 = float(np.abs(ham.coeffs).sum())
    sim = sv.StateVector(N, G, dtype)
    try:
        e, g, pt = sim.vqe_step(0, circ, params, ham, sv.LAZY, per_term=True)
        st = sim.last_stats
    finally:
        sim.close()
        del sim
        torch.cuda.empty_cache()
    assert st.qsu_qrs >= 1 and st.evc_qrs >= 1 and st.hpsi_passes >= 1 and st.adj_passes >= 1
    if dtype == sv.C64:
        tol_t, tol = 2e-5, 1e-4 * l1
    else:
        tol_t, tol = 1e-10, 1e-10 * l1
    assert np.max(np.abs(pt - terms)) < tol_t
    assert abs(e - energy) < tol
    assert np.max(np.abs(g - grad)) < tol
