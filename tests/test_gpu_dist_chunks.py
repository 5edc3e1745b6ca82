"""The per-chunk work of the sharded state (paper_2410_04252_gb300.dist) on
the GPU, through the C ABI, against the FP64 oracle on the same chunk:
a tile's gates with their targets mapped to physical local bits
(apply_local), and the strings' local sums (expect_local), whose global-bit
Z signs the orchestration applies.  Tolerances as in the parity tests."""
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
from paper_2410_04252_gb300 import dist as D  # noqa: E402


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_apply_local_and_expect_local(dtype):
    n, L = 12, 10
    circ = W.random_circuit(n, 60, 91, (W.RY, W.RZ, W.CZ, W.GIVENS, W.DEXC))
    params = W.uniform_params(circ.nparams, 92, 0.0, 2 * math.pi)
    # a layout that puts qubits 0..L-1 on physical bits in a scrambled order
    rng = W.SplitMix64(93)
    l2p = list(range(n))
    for i in range(L - 1, 0, -1):
        j = rng.randint(i + 1)
        l2p[i], l2p[j] = l2p[j], l2p[i]
    ids = [i for i in range(circ.m) if all(q < L for q in circ.targets(i))]
    rs = np.random.default_rng(94)
    host = rs.standard_normal(1 << L) + 1j * rs.standard_normal(1 << L)
    host /= np.linalg.norm(host)
    chunk = torch.tensor(host, dtype=dtype, device="cuda")
    start = chunk.cpu().numpy().astype(np.complex128)
    D.apply_local(chunk, L, circ, params, ids, l2p)
    loc = D.local_circuit(circ, ids, l2p)
    loc.n = L
    want = oracle.apply_circuit(start, loc, params)
    tol = 2e-5 if dtype == torch.complex64 else 1e-12
    assert np.max(np.abs(chunk.cpu().numpy() - want)) < tol
    ham = W.random_hamiltonian(L, 300, 95)
    x, z = W.pauli_masks(ham)
    got = D.expect_local(chunk, L, x, z)
    ref = oracle.expect_terms(chunk.cpu().numpy().astype(np.complex128), ham).real
    assert np.max(np.abs(got - ref)) < tol
    D.release_handles()
