"""Pins for the oracle gradients (oracle/grad.py): closed forms and the
agreement of two independent methods."""
import math

import numpy as np

from oracle import grad
from paper_2410_04252_gb300 import workloads as W


def test_closed_form_one_qubit():
    # RY(t) then RZ(p) on |0>: <X> = sin t cos p, <Z> = cos t
    c = W._circuit(1, [(W.RY, (0,), 0, -1), (W.RZ, (0,), 1, -1)], 2)
    h = W.Hamiltonian(1, np.array([[1], [3]], np.uint8), np.array([0.7, -1.3]))
    for t, p in [(0.4, 1.1), (-2.0, 0.3), (2.5, -2.9)]:
        params = np.array([t, p])
        e = grad.objective(c, params, h)
        assert abs(e - (0.7 * math.sin(t) * math.cos(p) - 1.3 * math.cos(t))) < 1e-14
        ref = np.array([0.7 * math.cos(t) * math.cos(p) + 1.3 * math.sin(t),
                        -0.7 * math.sin(t) * math.sin(p)])
        np.testing.assert_allclose(grad.parameter_shift(c, params, h), ref, atol=1e-14)
        np.testing.assert_allclose(grad.finite_difference(c, params, h), ref, atol=1e-9)


def test_shift_rule_matches_finite_differences():
    n = 6
    c = W.hea_circuit(n, 2)
    params = W.uniform_params(c.nparams, 5, 0, 2 * math.pi)
    h = W.random_hamiltonian(n, 20, 6)
    ps = grad.parameter_shift(c, params, h)
    fd = grad.finite_difference(c, params, h)
    assert not np.any(np.isnan(ps))
    np.testing.assert_allclose(ps, fd, atol=1e-8)


def test_fabric_shared_parameter_is_not_shiftable():
    c = W.fabric_circuit(8, 2)
    assert not grad.shiftable(c).any()
    params = W.uniform_params(c.nparams, 8, -math.pi, math.pi)
    h = W.jw_hamiltonian(8, 16, 3)
    init = W.half_filled_index(8)
    fd = grad.finite_difference(c, params, h, init)
    # a shared parameter's derivative is the sum over the gates that use it:
    # perturb it in one gate at a time (split the parameter) and add up
    gates = [(int(c.kinds[i]), c.targets(i), i, -1) for i in range(c.m)]
    split = W._circuit(8, gates, c.m)
    sp = np.array([params[int(c.param[i])] for i in range(c.m)])
    fds = grad.finite_difference(split, sp, h, init)
    summed = np.zeros(c.nparams)
    for i in range(c.m):
        summed[int(c.param[i])] += fds[i]
    np.testing.assert_allclose(fd, summed, atol=1e-8)
