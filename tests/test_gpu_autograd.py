"""torch.autograd.Function over the adjoint gradient, on the n=14 copy of the
n=32 workload (HEA 6 layers, 1024 random strings): against the oracle's
parameter-shift rule and central finite differences on a seeded sample of
parameters, and the energy against the oracle."""
import math

import numpy as np
import pytest

from oracle import grad as ograd
from paper_2410_04252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
sv = pytest.importorskip("paper_2410_04252_gb300.sv")
ag = pytest.importorskip("paper_2410_04252_gb300.autograd")


def test_autograd_matches_parameter_shift_and_fd_n14_copy():
    cfg = W.CONFIGS[3]
    n = cfg["n_small"]
    circ = W.make_circuit(cfg, n)
    params = W.make_params(3, circ)
    ham = W.make_hamiltonian(3, n)
    l1 = float(np.abs(ham.coeffs).sum())
    sim = sv.StateVector(n, cfg["g"], sv.C64)
    theta = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    e = ag.vqe_energy(theta, sim, circ, ham, sv.LAZY, 0)
    e.backward()
    g = theta.grad.numpy()
    assert abs(e.item() - ograd.objective(circ, params, ham)) < 1e-4 * l1
    rng = W.SplitMix64(77)
    sample = sorted({rng.randint(circ.nparams) for _ in range(40)})
    ps = ograd.parameter_shift(circ, params, ham, which=sample)
    fd = ograd.finite_difference(circ, params, ham, which=sample)
    for p in sample:
        assert abs(g[p] - ps[p]) < 1e-4 * l1
        assert abs(g[p] - fd[p]) < 1e-4 * l1
    # the eager schedule gives the same gradient
    sim.reset(0)
    e2, g2 = sim.grad(circ, params, ham, sv.EAGER)
    assert np.max(np.abs(g2 - g)) < 1e-4 * l1


def test_autograd_descent_lowers_energy():
    n = 8
    circ = W.hea_circuit(n, 2)
    ham = W.random_hamiltonian(n, 24, 5)
    sim = sv.StateVector(n, 2, sv.C64)
    theta = torch.tensor(W.uniform_params(circ.nparams, 6, 0, 2 * math.pi), requires_grad=True)
    opt = torch.optim.SGD([theta], lr=0.05)
    energies = []
    for _ in range(15):
        opt.zero_grad()
        e = ag.vqe_energy(theta, sim, circ, ham)
        e.backward()
        opt.step()
        energies.append(e.item())
    assert energies[-1] < energies[0]
