"""sv_expect_noalloc (no device allocation; scratch in a static device array)
against the ordinary sv_expect, through the C ABI, on two calls in a row, and
against the FP64 oracle from small n (fewer cosets than CTAs) up to the
256-string limit.  Collected last so that a failure here leaves every other
test already run."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2410_04252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
sv = pytest.importorskip("paper_2410_04252_gb300.sv")


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
def test_noalloc_matches_expect_two_calls(dtype):
    n = 14
    circ = W.hea_circuit(n, 3)
    params = W.uniform_params(circ.nparams, 41, 0.0, 2 * math.pi)
    hA = W.random_hamiltonian(n, 200, 42)
    hB = W.jw_hamiltonian(n, 256, 43)
    sim = sv.StateVector(n, 0, dtype)        # no virtual chunks: the layout stays the index order
    sim.reset(0)
    sim.apply_circuit(circ, params, sv.LAZY)
    assert list(sim.permutation()) == list(range(n))
    tol_t = 2e-5 if dtype == sv.C64 else 1e-12
    refs = {}
    for name, h in (("A", hA), ("B", hB)):
        e, pt = sim.expect(h, sv.LAZY, keep_layout=True)
        refs[name] = (e, pt, float(np.abs(h.coeffs).sum()))
    # A, A, B, A: two calls in a row, then a different call, then A again
    for name, h in (("A", hA), ("A", hA), ("B", hB), ("A", hA)):
        paulis, coeffs = sv.hamiltonian_arrays(h)
        e, pt = sv.expect_noalloc(sim.state, n, dtype, paulis, coeffs)
        e_ref, pt_ref, l1 = refs[name]
        assert abs(e - e_ref) < (1e-4 * l1 if dtype == sv.C64 else 1e-11)
        assert np.max(np.abs(pt - pt_ref)) < tol_t


def test_noalloc_rejects_oversize_calls():
    n = 10
    sim = sv.StateVector(n, 0, sv.C64)
    sim.reset(0)
    h = W.random_hamiltonian(n, 257, 44)
    paulis, coeffs = sv.hamiltonian_arrays(h)
    with pytest.raises(sv.SvError) as e:
        sv.expect_noalloc(sim.state, n, sv.C64, paulis, coeffs)
    assert e.value.status == sv.SV_EINVAL and "256" in str(e.value)


def _random_state(n, seed, dtype):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.linalg.norm(v)
    t = torch.tensor(v, dtype=torch.complex64 if dtype == sv.C64 else torch.complex128, device="cuda")
    # the oracle sees exactly the amplitudes the GPU holds (complex64 rounding included)
    return t, t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("dtype", [sv.C64, sv.C128])
@pytest.mark.parametrize("n", [1, 3, 6, 9, 14])
def test_noalloc_matches_oracle(n, dtype):
    """Per-term values and energy against the oracle's per-string sum; n = 14
    takes the 256-string maximum (random and Jordan-Wigner-shaped strings)."""
    state, host = _random_state(n, 500 + n, dtype)
    hams = [W.random_hamiltonian(n, 256 if n == 14 else 40, 600 + n)]
    if n >= 2:
        hams.append(W.jw_hamiltonian(n, 256 if n == 14 else 40, 700 + n))
    tol_t = 2e-5 if dtype == sv.C64 else 1e-12
    for h in hams:
        ref = oracle.expect_terms(host, h)
        assert np.max(np.abs(ref.imag)) < 1e-12
        paulis, coeffs = sv.hamiltonian_arrays(h)
        for _ in range(2):                       # two calls in a row share the array
            e, pt = sv.expect_noalloc(state, n, dtype, paulis, coeffs)
            assert np.max(np.abs(pt - ref.real)) < tol_t
            l1 = float(np.abs(h.coeffs).sum())
            assert abs(e - float(h.coeffs @ ref.real)) < (1e-4 * l1 if dtype == sv.C64 else 1e-11)


def test_noalloc_rejects_unaligned_or_misshapen_state():
    n = 8
    state, _ = _random_state(n + 1, 11, sv.C64)
    h = W.random_hamiltonian(n, 8, 12)
    paulis, coeffs = sv.hamiltonian_arrays(h)
    e = ctypes.c_double(0.0)
    # a complex64 view one element in: 8-byte aligned only; refused before any launch
    st = sv._lib.sv_expect_noalloc(ctypes.c_void_p(state.data_ptr() + 8), n, sv.C64,
                                   sv._ptr(paulis), sv._ptr(coeffs), len(coeffs), ctypes.byref(e), None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sv.SV_EINVAL and "aligned" in sv._lib.sv_last_error().decode()
    with pytest.raises(sv.SvError) as err:                                    # the same through the binding
        sv.expect_noalloc(state[1:1 + (1 << n)], n, sv.C64, paulis, coeffs)
    assert err.value.status == sv.SV_EINVAL
    with pytest.raises(ValueError):
        sv.expect_noalloc(state, n, sv.C64, paulis, coeffs)                   # 2^(n+1) amplitudes
    with pytest.raises(ValueError):
        sv.expect_noalloc(state[: 1 << n], n, sv.C128, paulis, coeffs)        # wrong dtype
