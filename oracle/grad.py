"""CPU ORACLE -- test infrastructure, not part of the product.

Gradients of the VQE objective E(theta) = <psi0|U(theta)^dagger H U(theta)|psi0>
(Eqs. vqe, vqe_qsu, vqe_evc), computed only from repeated forward
evaluations of the plain simulator -- never by an adjoint sweep, so that the
library's adjoint kernel is checked against an independent method.

  parameter_shift: for a parameter that enters exactly one gate whose
    generator has eigenvalues +-1 (RY, RZ, since U = exp(-i theta G/2)),
    dE/dtheta = (E(theta + pi/2) - E(theta - pi/2)) / 2 exactly.
  finite_difference: central differences (E(theta+h) - E(theta-h)) / (2h),
    any parameter, truncation error O(h^2).

Pinned by tests/test_oracle_grad.py: a one-qubit closed form
(E = cos(theta) for <Z> after RY(theta)), agreement of the two methods, and
the shift rule against finite differences on random circuits.
"""
from __future__ import annotations

import math

import numpy as np

from . import apply_circuit, basis_state, energy

RY, RZ = 0, 1


def objective(circ, params, ham, init_index: int = 0) -> float:
    psi = apply_circuit(basis_state(circ.n, init_index), circ, params)
    return energy(psi, ham)


def finite_difference(circ, params, ham, init_index: int = 0, h: float = 1e-5, which=None) -> np.ndarray:
    params = np.asarray(params, np.float64)
    idx = range(len(params)) if which is None else which
    g = np.zeros(len(params))
    for p in idx:
        up = params.copy(); up[p] += h
        dn = params.copy(); dn[p] -= h
        g[p] = (objective(circ, up, ham, init_index) - objective(circ, dn, ham, init_index)) / (2 * h)
    return g


def shiftable(circ) -> np.ndarray:
    """Boolean per parameter: True if it drives exactly one RY/RZ gate."""
    uses = np.zeros(circ.nparams, np.int64)
    ok = np.ones(circ.nparams, bool)
    for i in range(circ.m):
        p = int(circ.param[i])
        if p < 0:
            continue
        uses[p] += 1
        if int(circ.kinds[i]) not in (RY, RZ):
            ok[p] = False
    return ok & (uses == 1)


def parameter_shift(circ, params, ham, init_index: int = 0, which=None) -> np.ndarray:
    """Two-term shift rule; NaN for parameters it does not apply to."""
    params = np.asarray(params, np.float64)
    ok = shiftable(circ)
    idx = range(len(params)) if which is None else which
    g = np.full(len(params), np.nan)
    for p in idx:
        if not ok[p]:
            continue
        up = params.copy(); up[p] += math.pi / 2
        dn = params.copy(); dn[p] -= math.pi / 2
        g[p] = 0.5 * (objective(circ, up, ham, init_index) - objective(circ, dn, ham, init_index))
    return g
