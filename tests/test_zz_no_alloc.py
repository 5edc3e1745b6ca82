"""sv_expect_noalloc (no device allocation; scratch in a static device array)
against the ordinary sv_expect, through the C ABI, on two calls in a row.
Collected last so that a failure here leaves every other test already run."""
import math

import numpy as np
import pytest

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
