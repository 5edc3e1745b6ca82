"""Autotuner and the options it searches (tile size k, fusion depth, coset
pass shape, batched CTA size): whatever they are set to, results stay those
of the FP64 oracle (same tolerances as the parity tests)."""
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


def l1(h):
    return float(np.abs(h.coeffs).sum())


@pytest.mark.parametrize("tile_bits,fuse_max", [(9, 0), (10, 3), (11, 1), (12, 16), (13, 0)])
def test_options_keep_parity(tile_bits, fuse_max):
    n, g = 14, 3
    c = W.hea_circuit(n, 3)
    p = W.uniform_params(c.nparams, 41, 0, 2 * math.pi)
    ham = W.random_hamiltonian(n, 48, 43)
    s = sv.StateVector(n, g, sv.C64)
    o = s.options()
    o.tile_bits, o.fuse_max = tile_bits, fuse_max
    o.low_bits = min(o.low_bits, tile_bits - 4)
    s.set_options(o)
    e, grad, _ = s.vqe_step(0, c, p, ham, sv.LAZY)
    tol = 1e-4 * l1(ham)
    assert abs(e - ograd.objective(c, p, ham)) < tol
    assert np.max(np.abs(grad - ograd.parameter_shift(c, p, ham))) < tol
    if fuse_max:
        plan = sv.plan_qsu(n, g, c, sv.LAZY, o)
        assert max(len(ps["ops"]) for ps in plan["passes"]) <= fuse_max


def test_autotune_vqe_step():
    n, g = 15, 3
    c = W.hea_circuit(n, 2)
    p = W.uniform_params(c.nparams, 51, 0, 2 * math.pi)
    ham = W.random_hamiltonian(n, 64, 53)
    s = sv.StateVector(n, g, sv.C64)
    best, ms = s.autotune(c, p, ham, sv.LAZY, reps=1)
    assert ms > 0
    assert 8 <= best.tile_bits <= 13 and best.fuse_max >= 0
    o = s.options()
    assert (o.tile_bits, o.fuse_max, o.evc_low_bits, o.evc_span) == \
        (best.tile_bits, best.fuse_max, best.evc_low_bits, best.evc_span)
    e, grad, _ = s.vqe_step(0, c, p, ham, sv.LAZY)
    tol = 1e-4 * l1(ham)
    assert abs(e - ograd.objective(c, p, ham)) < tol
    assert np.max(np.abs(grad - ograd.parameter_shift(c, p, ham))) < tol


def test_autotune_qsu_only():
    n, g = 14, 2
    c = W.fabric_circuit(n, 4)
    p = W.uniform_params(c.nparams, 61, -math.pi, math.pi)
    init = (1 << (n // 2)) - 1
    s = sv.StateVector(n, g, sv.C64)
    best, ms = s.autotune(c, p, None, sv.LAZY, init_index=init, reps=1)
    assert ms > 0
    s.reset(init)
    s.apply_circuit(c, p, sv.LAZY)
    ref = oracle.apply_circuit(oracle.basis_state(n, init), c, p)
    assert np.max(np.abs(s.get_state() - ref)) < 2e-5


@pytest.mark.parametrize("tile_bits,threads", [(10, 256), (11, 512), (12, 256), (12, 512), (13, 512)])
def test_batch_options_keep_parity(tile_bits, threads):
    n = 11
    out = W.batch_states(10, n, 4, 1)
    circs = [W.hea_circuit(n, layers) for layers, _ in out]
    params = [pp for _, pp in out]
    ham = W.random_hamiltonian(n, 40, 77)
    o = sv.default_options(sv.C64)
    o.tile_bits, o.threads = tile_bits, threads
    o.low_bits = min(o.low_bits, tile_bits - 4)
    e, gl, _, _ = sv.batch_run(n, sv.C64, circs, params, ham, options=o)
    tol = 1e-4 * l1(ham)
    for b in range(len(circs)):
        assert abs(e[b] - ograd.objective(circs[b], params[b], ham)) < tol
    for b in (0, 9):
        assert np.max(np.abs(gl[b] - ograd.parameter_shift(circs[b], params[b], ham))) < tol


def test_batch_autotune():
    n = 12
    out = W.batch_states(24, n, 5, 2)
    circs = [W.hea_circuit(n, layers) for layers, _ in out]
    params = [pp for _, pp in out]
    ham = W.random_hamiltonian(n, 64, 79)
    best, ms = sv.batch_autotune(n, sv.C64, circs, params, ham, reps=1)
    assert ms > 0 and best.threads in (256, 512) and 10 <= best.tile_bits <= 13
    e, _, _, _ = sv.batch_run(n, sv.C64, circs, params, ham, options=best)
    e0, _, _, _ = sv.batch_run(n, sv.C64, circs, params, ham)
    assert np.max(np.abs(e - e0)) < 1e-4 * l1(ham)


def test_batch_rejects_unbuilt_shape():
    n = 10
    out = W.batch_states(2, n, 2, 1)
    circs = [W.hea_circuit(n, layers) for layers, _ in out]
    params = [pp for _, pp in out]
    ham = W.random_hamiltonian(n, 8, 3)
    o = sv.default_options(sv.C64)
    o.tile_bits, o.threads = 13, 256          # 32 amplitudes per thread: not built
    with pytest.raises(sv.SvError):
        sv.batch_run(n, sv.C64, circs, params, ham, options=o)


@pytest.mark.parametrize("n,g,nterms,kind", [(10, 3, 40, "random"), (14, 4, 64, "jw"), (20, 5, 160, "random"),
                                            (32, 6, 1024, "random"), (30, 6, 4096, "jw")])
def test_alg6_search_on_device_matches_host(n, g, nterms, kind):
    """The device search of Alg. 6 (one greedy step per launch, first maximum
    in lexicographic order) gives the host search's plan bit for bit."""
    h = W.random_hamiltonian(n, nterms, 5 + n) if kind == "random" else W.jw_hamiltonian(n, nterms, 5 + n)
    x, z = W.pauli_masks(h)
    od = sv.default_options(sv.C64)
    od.plan_device = 1
    oh = sv.default_options(sv.C64)
    oh.plan_device = 2
    pd = sv.plan_evc(n, g, x, z, sv.LAZY, od)
    ph = sv.plan_evc(n, g, x, z, sv.LAZY, oh)
    assert pd["order"] == ph["order"]
    assert [(t["begin"], t["end"], t["local_mask"], t["pairs"]) for t in pd["tiles"]] == \
        [(t["begin"], t["end"], t["local_mask"], t["pairs"]) for t in ph["tiles"]]
