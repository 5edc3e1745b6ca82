"""CPU ORACLE -- test infrastructure, not part of the product.

Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
its reference arm) may import this package.  It shares no code with the CUDA
library and never imports it.

Contents:
  svsim.c    plain FP64 gate-by-gate simulator and per-string EVC (Sec. III,
             Eqs. update_sv_gate, pauli_matrix, evc), built with gcc.
  planner.py the paper's scheduling algorithms written out step by step
             (Alg. 1-6, diagonalization of Eq. without_QR, the ad hoc rule).
  grad.py    parameter-shift and central finite-difference gradients of
             E(theta) = <psi0|U^dagger H U|psi0> (Eqs. vqe_qsu, vqe_evc).

Parity status per function is listed in the module docstrings; every function
here is pinned by tests/test_oracle_*.py against closed forms, brute-force
dense matrices or the paper's worked examples, except the ad hoc (eager) QR
rule, whose exact form the paper does not give ("parity unpinned" beyond its
definition and invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile svsim.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "svsim.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            L.osim_apply.restype = ctypes.c_int
            L.osim_apply.argtypes = [f64p, ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p,
                                     f64p, f64p, ctypes.c_int]
            L.osim_expect.restype = None
            L.osim_expect.argtypes = [f64p, ctypes.c_int, ctypes.c_int, u8p, f64p]
            L.osim_apply_hamiltonian.restype = None
            L.osim_apply_hamiltonian.argtypes = [f64p, ctypes.c_int, ctypes.c_int, u8p, f64p, f64p]
            L.osim_gate_matrix.restype = ctypes.c_int
            L.osim_gate_matrix.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_int, f64p]
            _lib = L
    return _lib


def basis_state(n: int, index: int) -> np.ndarray:
    """|index> as a complex128 vector."""
    psi = np.zeros(1 << n, np.complex128)
    psi[index] = 1.0
    return psi


def apply_circuit(psi: np.ndarray, circ, params, inverse: bool = False) -> np.ndarray:
    """U psi (or U^dagger psi) for `circ` (workloads.Circuit), gate by gate in
    the given order.  Returns a new complex128 vector."""
    out = np.ascontiguousarray(psi, np.complex128).copy()
    buf = out.view(np.float64)
    n = circ.n
    params = np.ascontiguousarray(params if params is not None and len(params) else np.zeros(1), np.float64)
    mats = np.ascontiguousarray(circ.mats if circ.mats.size else np.zeros(2), np.float64)
    rc = lib().osim_apply(buf, n, circ.m, np.ascontiguousarray(circ.kinds, np.int32),
                          np.ascontiguousarray(circ.qubits.reshape(-1), np.int32),
                          np.ascontiguousarray(circ.param, np.int32),
                          np.ascontiguousarray(circ.mat, np.int32), params, mats,
                          1 if inverse else 0)
    if rc != 0:
        raise ValueError("oracle: invalid gate list")
    return out


def expect_terms(psi: np.ndarray, ham) -> np.ndarray:
    """Complex <psi|P_t|psi> for every string t (workloads.Hamiltonian)."""
    psi = np.ascontiguousarray(psi, np.complex128)
    n = ham.n
    out = np.zeros(2 * ham.nterms, np.float64)
    lib().osim_expect(psi.view(np.float64), n, ham.nterms,
                      np.ascontiguousarray(ham.letters.reshape(-1), np.uint8), out)
    return out[0::2] + 1j * out[1::2]


def energy(psi: np.ndarray, ham) -> float:
    """E = sum_t a_t <psi|P_t|psi> (Eq. evc); the a_t are real."""
    return float(np.dot(ham.coeffs, expect_terms(psi, ham).real))


def apply_hamiltonian(psi: np.ndarray, ham) -> np.ndarray:
    """H psi = sum_t a_t P_t psi as a vector."""
    psi = np.ascontiguousarray(psi, np.complex128)
    out = np.zeros_like(psi)
    lib().osim_apply_hamiltonian(psi.view(np.float64), ham.n, ham.nterms,
                                 np.ascontiguousarray(ham.letters.reshape(-1), np.uint8),
                                 np.ascontiguousarray(ham.coeffs, np.float64), out.view(np.float64))
    return out


def gate_matrix(kind: int, theta: float = 0.0, mat=None, inverse: bool = False) -> np.ndarray:
    """The dense matrix the oracle applies for one gate (complex, dim x dim)."""
    u = np.zeros(2 * 16 * 16, np.float64)
    mp = None
    if mat is not None:
        mat = np.ascontiguousarray(mat, np.float64)
        mp = mat.ctypes.data_as(ctypes.c_void_p)
    dim = lib().osim_gate_matrix(kind, float(theta), mp, 1 if inverse else 0, u)
    if dim < 0:
        raise ValueError("oracle: bad gate kind")
    return (u[0:2 * dim * dim:2] + 1j * u[1:2 * dim * dim:2]).reshape(dim, dim)
