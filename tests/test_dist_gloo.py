"""The sharded state (paper_2410_04252_gb300.dist) on CPU gloo ranks, one
process per rank as torchrun starts them.

* qr_exchange on 2 and 4 ranks equals, bit for bit, the single-buffer QR:
  amplitude x moves to x with bits a_i and g_i exchanged (Sec. III-B-4).
* sharded_energy (lazy QSU tile by tile with its QRs as exchanges, lazy EVC
  with per-chunk Z signs and a sum over ranks) equals the FP64 oracle: the
  final state bit for bit against the oracle applying the same gate order to
  one buffer and permuting it to the final layout, and the energy and every
  string's value within 1e-12.  The work on a chunk runs in the library's
  CUDA kernels on a GPU rank; on these CPU ranks the test hands it to the
  oracle (same definition of a gate and a string on the chunk's qubits).
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("paper_2410_04252_gb300.sv")   # the host planner (no CUDA call)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, target, args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda v: v[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return got


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _swap_bits(x, pairs):
    for a, b in pairs:
        if ((x >> a) ^ (x >> b)) & 1:
            x ^= (1 << a) | (1 << b)
    return x


def _state(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)


def _exchange_rank(rank, world, port, q, n, pairs_list):
    dist = _init(rank, world, port)
    try:
        from paper_2410_04252_gb300 import dist as D
        L = n - (world.bit_length() - 1)
        psi = _state(n, 7)
        chunk = torch.from_numpy(psi[rank << L:(rank + 1) << L].copy())
        for pairs in pairs_list:
            D.qr_exchange(chunk, L, rank, pairs)
        q.put((rank, chunk.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,pairs_list", [
    (2, [[(2, 5)], [(0, 5)], [(4, 5)]]),
    (4, [[(1, 6)], [(3, 7), (0, 6)], [(5, 7)], [(0, 6), (2, 7)]]),
])
def test_qr_exchange_is_the_bit_swap(world, pairs_list):
    n = 8 if world == 4 else 6
    got = _run(world, _exchange_rank, (n, pairs_list))
    sharded = np.concatenate([c for _, c in got])
    psi = _state(n, 7)
    want = psi.copy()
    for pairs in pairs_list:
        nxt = np.empty_like(want)
        for x in range(1 << n):
            nxt[_swap_bits(x, pairs)] = want[x]
        want = nxt
    assert np.array_equal(sharded, want)


def _letters(x, z, n):
    """Pauli letters (0 I, 1 X, 2 Y, 3 Z) per qubit of masks x, z."""
    out = np.zeros((len(x), n), np.uint8)
    for t, (xv, zv) in enumerate(zip(x, z)):
        for b in range(n):
            xb, zb = (int(xv) >> b) & 1, (int(zv) >> b) & 1
            out[t, b] = 2 if xb and zb else 1 if xb else 3 if zb else 0
    return out


def _energy_rank(rank, world, port, q, n, layers, nterms, intra_bits=0):
    dist = _init(rank, world, port)
    try:
        import oracle
        from paper_2410_04252_gb300 import dist as D
        from paper_2410_04252_gb300 import workloads as W

        def apply_cpu(chunk, L, circ, params, gate_ids, l2p):
            if len(gate_ids) == 0:
                return
            c = D.local_circuit(circ, gate_ids, l2p)
            c.n = L
            chunk.copy_(torch.from_numpy(oracle.apply_circuit(chunk.numpy(), c, params)))

        def expect_cpu(chunk, L, x, z):
            h = W.Hamiltonian(L, _letters(x, z, L), np.ones(len(x)))
            return oracle.expect_terms(chunk.numpy(), h).real

        D.apply_local = apply_cpu
        D.expect_local = expect_cpu
        circ = W.hea_circuit(n, layers)
        params = W.uniform_params(circ.nparams, 31, 0.0, 2 * np.pi)
        ham = _narrow_hamiltonian(n, nterms, n - (world.bit_length() - 1))
        L = n - (world.bit_length() - 1)
        chunk = torch.zeros(1 << L, dtype=torch.complex128)
        if intra_bits:
            from paper_2410_04252_gb300 import sv
            o = sv.default_options()
            o.intra_bits = intra_bits
            e, vals, l2p = D.sharded_energy(n, circ, params, ham, chunk, schedule=sv.HIER, options=o)
        else:
            e, vals, l2p = D.sharded_energy(n, circ, params, ham, chunk)
        q.put((rank, e, vals, l2p, chunk.numpy().copy()))
    finally:
        dist.destroy_process_group()


def _narrow_hamiltonian(n, nterms, nL):
    """Random strings (each qubit I/X/Y/Z) with at most nL X/Y letters."""
    from paper_2410_04252_gb300 import workloads as W
    h = W.random_hamiltonian(n, 3 * nterms, 44)
    keep = [t for t in range(h.nterms) if int(np.sum((h.letters[t] == 1) | (h.letters[t] == 2))) <= nL][:nterms]
    return W.Hamiltonian(n, h.letters[keep].copy(), h.coeffs[keep].copy())


@pytest.mark.parametrize("world,intra_bits", [(2, 0), (4, 0), (4, 1)])
def test_sharded_energy_matches_single_buffer(world, intra_bits):
    """Lazy plan on 2 and 4 ranks; hierarchical plan (Alg. 4/5) on 4 ranks
    with one global qubit inside a node."""
    import oracle
    from paper_2410_04252_gb300 import sv
    from paper_2410_04252_gb300 import workloads as W
    n, layers, nterms = 8, 3, 40
    got = _run(world, _energy_rank, (n, layers, nterms, intra_bits))
    energies = [v[1] for v in got]
    assert max(energies) == min(energies)            # every rank holds the reduced result
    e, vals, l2p = got[0][1], got[0][2], got[0][3]
    sharded = np.concatenate([v[4] for v in got])
    circ = W.hea_circuit(n, layers)
    params = W.uniform_params(circ.nparams, 31, 0.0, 2 * np.pi)
    ham = _narrow_hamiltonian(n, nterms, n - (world.bit_length() - 1))
    # single buffer, the plan's gate order, then the final layout's permutation
    if intra_bits:
        o = sv.default_options()
        o.intra_bits = intra_bits
        plan = sv.plan_qsu(n, world.bit_length() - 1, circ, sv.HIER, o)
    else:
        plan = sv.plan_qsu(n, world.bit_length() - 1, circ, sv.LAZY)
    order = plan["order"]
    assert any(t["pairs"] for t in plan["tiles"])           # the exchange ran
    c = W.Circuit(n, circ.kinds[order], circ.qubits[order], circ.param[order], circ.mat[order], circ.nparams)
    psi = oracle.apply_circuit(oracle.basis_state(n, 0), c, params)
    phys = np.empty_like(psi)
    for x in range(1 << n):
        y = 0
        for qb in range(n):
            if (x >> qb) & 1:
                y |= 1 << l2p[qb]
        phys[y] = psi[x]
    assert np.array_equal(sharded, phys)
    ref = oracle.expect_terms(oracle.apply_circuit(oracle.basis_state(n, 0), circ, params), ham).real
    assert np.max(np.abs(vals - ref)) < 1e-12
    assert abs(e - float(ham.coeffs @ ref)) < 1e-12


def test_comm_cost_of_fig9():
    """Eq. comm_cost on the hierarchical plan of Fig. 9 (2 inter and 3 intra
    QRs), with weights from link bandwidths (one QR of s pairs moves 1 - 2^-s
    of a rank's chunk)."""
    from paper_2410_04252_gb300 import dist as D
    from paper_2410_04252_gb300 import sv
    from paper_2410_04252_gb300 import workloads as W
    n, nL = 16, 12
    c = W.fabric_blocks_circuit(n, 12)
    o = sv.default_options()
    o.intra_bits = 2
    plan = sv.plan_qsu(n, n - nL, c, sv.HIER, o)
    assert D.qr_kinds(plan, n) == ["inter", "intra", "intra", "inter", "intra"]
    assert D.comm_cost(plan, n, 1.0, 20.0) == 2 * 20.0 + 3 * 1.0
    w = D.qr_weight(30, 5, 2, 16, 100.0)
    assert w == pytest.approx(0.75 * (1 << 25) * 16 / 100e9)
    flat = sv.plan_qsu(n, n - nL, c, sv.LAZY)
    assert D.qr_kinds(flat, n) == ["inter"] * 3     # no intra set: every QR crosses nodes


def test_qr_exchange_rejects_pairs_that_are_not_local_global():
    """A QR pair must be (local bit < L, global bit >= L); anything else is
    refused before any data moves."""
    from paper_2410_04252_gb300 import dist as D
    chunk = torch.zeros(1 << 4, dtype=torch.complex128)
    for pairs in ([(4, 5)], [(1, 3)], [(-1, 5)]):
        with pytest.raises(ValueError):
            D.qr_exchange(chunk, 4, 0, pairs)
    D.qr_exchange(chunk, 4, 0, [])           # no pairs: nothing to do


def test_comm_cost_counts_only_qrs():
    """A plan without QRs costs nothing; weights scale the two QR kinds."""
    from paper_2410_04252_gb300 import dist as D
    plan = {"tiles": [{"local_mask": 0xFF, "pairs": []}]}
    assert D.qr_kinds(plan, 10) == [] and D.comm_cost(plan, 10, 1.0, 5.0) == 0.0
    plan = {"tiles": [{"local_mask": 0xFF, "pairs": []},
                      {"local_mask": 0x1FE, "pairs": [(0, 8)], "intra_mask": 0x200},
                      {"local_mask": 0x3FC, "pairs": [(1, 9)], "intra_mask": 0x002}]}
    # the first QR changes the inter set {8, 9} -> {0}; the second swaps a
    # local qubit with the intra one and leaves the inter set {0} alone
    assert D.qr_kinds(plan, 10) == ["inter", "intra"]
    assert D.comm_cost(plan, 10, 2.0, 7.0) == 9.0
