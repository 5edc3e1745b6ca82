"""The persistent batched kernel (sv_batch_run) against the FP64 oracle and
against the single-state path, on seeded independent states of different
depths sharing one Hamiltonian."""
import math

import numpy as np
import pytest

import oracle
from oracle import grad as ograd
from paper_2410_04252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
sv = pytest.importorskip("paper_2410_04252_gb300.sv")


def states(n, count, max_layers, min_layers=1):
    out = W.batch_states(count, n, max_layers, min_layers)
    circs = [W.hea_circuit(n, layers) for layers, _ in out]
    return circs, [p for _, p in out]


@pytest.mark.parametrize("dtype,n", [(sv.C64, 10), (sv.C64, 14), (sv.C128, 9)])
def test_batch_matches_oracle(dtype, n):
    circs, params = states(n, 12, 4)
    ham = W.random_hamiltonian(n, 40, 71 + n)
    l1 = float(np.abs(ham.coeffs).sum())
    e, g, t, st = sv.batch_run(n, dtype, circs, params, ham)
    tol = 1e-4 * l1 if dtype == sv.C64 else 1e-10
    for b in range(len(circs)):
        assert abs(e[b] - ograd.objective(circs[b], params[b], ham)) < tol
    for b in (0, 5, 11):
        ps = ograd.parameter_shift(circs[b], params[b], ham)
        assert np.max(np.abs(g[b] - ps)) < tol
    assert np.all(t[:, 1] >= t[:, 0])
    assert st.launches == 1


def test_batch_matches_single_state_path_and_mixed_circuits():
    n = 12
    circs, params = states(n, 20, 6, 2)
    # a fabric circuit and a random circuit with fixed matrices-free gates in the mix
    fc = W.fabric_circuit(n, 3)
    circs.append(fc)
    params.append(W.uniform_params(fc.nparams, 5, -math.pi, math.pi))
    rc = W.random_circuit(n, 50, 9)
    circs.append(rc)
    params.append(W.uniform_params(rc.nparams, 6, -2, 2))
    ham = W.jw_hamiltonian(n, 96, 12)
    l1 = float(np.abs(ham.coeffs).sum())
    e, g, t, st = sv.batch_run(n, sv.C64, circs, params, ham)
    sim = sv.StateVector(n, 0, sv.C64)
    for b in range(len(circs)):
        sim.reset(0)
        e1, g1 = sim.grad(circs[b], params[b], ham, sv.LAZY)
        assert abs(e[b] - e1) < 1e-4 * l1
        assert np.max(np.abs(g[b] - g1)) < 1e-4 * l1


def test_batch_rejects_bad_input():
    n = 8
    circs, params = states(n, 2, 2)
    ham = W.random_hamiltonian(n, 10, 1)
    bad = W._circuit(n, [(W.RY, (n + 1,), 0, -1)], 1)
    with pytest.raises(sv.SvError):
        sv.batch_run(n, sv.C64, [bad], [np.zeros(1)], ham)
    with pytest.raises(sv.SvError):
        sv.batch_run(30, sv.C64, circs, params, W.random_hamiltonian(30, 4, 1))
