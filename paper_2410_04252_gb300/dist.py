"""The state sharded over ranks, one chunk per rank (the paper's p-SVQCS
layout, Sec. III-B): physical index bits L..n-1 (the global qubits) are the
rank index, bits 0..L-1 index the rank's chunk of 2^L amplitudes.

  qr_exchange     a qubit reordering (Sec. III-B-4) as a pairwise exchange:
                  swapping local bit a with global bit g moves every amplitude
                  whose bit a differs from the rank's bit g to the rank that
                  differs in g, at the position that differs in a; for s pairs
                  at once each rank swaps 2^s - 1 sub-blocks of 2^(L-s)
                  amplitudes with 2^s - 1 partners (the all-to-all of a QR);
  allreduce_sum   the EVC reduction over ranks (Eq. parallel_evc);
  sharded_energy  lazy QSU (Alg. 1-3) then lazy EVC (Alg. 6), tile by tile:
                  the QR before a tile, then the tile's work on every chunk.

Data moves with torch.distributed point-to-point operations (NCCL between
GPUs, gloo between CPU processes).  The work on a chunk runs in the
library's CUDA kernels through the C ABI (apply_local, expect_local): a
handle of L qubits attached to the chunk applies the tile's gates with their
targets mapped to physical local bits, and the allocation-free expectation
entry point evaluates the tile's strings on the local bits, signed by the
global bits of Z letters (the per-chunk sign of Eq. par_exp).
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def _bit_view(chunk, L: int, bits: list[int]):
    """A view of the 2^L chunk with one size-2 dimension per bit of `bits`
    (and the runs between them as dimensions of their own); returns the view
    and, per bit (in the order given), its dimension."""
    order = sorted(bits, reverse=True)
    shape, dim_of, prev = [], {}, L
    for b in order:
        shape.append(1 << (prev - b - 1))
        dim_of[b] = len(shape)
        shape.append(2)
        prev = b
    shape.append(1 << prev)
    return chunk.view(*shape), [dim_of[b] for b in bits]


def _sub_block(view, dims: list[int], values: list[int]):
    idx = [slice(None)] * view.dim()
    for d, v in zip(dims, values):
        idx[d] = v
    return view[tuple(idx)]


def qr_exchange(chunk, L: int, rank: int, pairs, group=None) -> None:
    """Apply the QR that swaps physical bits (a_i, g_i) (a_i < L <= g_i) to
    the sharded state, in place on this rank's chunk.  The sub-block B_e
    (local bits a_i equal to e_i) goes to the rank whose bits g_i - L are e,
    and the block that rank holds at e = this rank's bits g_i - L comes back
    into B_e; the sub-block with e equal to this rank's bits stays."""
    import torch.distributed as dist
    if not pairs:
        return
    a_bits = [int(a) for a, _ in pairs]
    r_bits = [int(g) - L for _, g in pairs]
    if any(a >= L or a < 0 for a in a_bits) or any(b < 0 for b in r_bits):
        raise ValueError("qr_exchange: pairs must be (local bit, global bit)")
    own = [(rank >> b) & 1 for b in r_bits]
    view, dims = _bit_view(chunk, L, a_bits)
    ops, moves = [], []
    for e in range(1 << len(pairs)):
        ev = [(e >> i) & 1 for i in range(len(pairs))]
        if ev == own:
            continue
        peer = rank
        for b, v in zip(r_bits, ev):
            peer = (peer & ~(1 << b)) | (v << b)
        blk = _sub_block(view, dims, ev)
        send = blk.contiguous()
        recv = send.new_empty(send.shape)
        ops.append(dist.P2POp(dist.isend, send, peer, group))
        ops.append(dist.P2POp(dist.irecv, recv, peer, group))
        moves.append((blk, recv))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    for blk, recv in moves:
        blk.copy_(recv)


def allreduce_sum(values, group=None, device=None):
    """Sum of every rank's values (FP64 host array in, same shape out); the
    reduction runs on `device` (a CUDA device for NCCL, the host for gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(values, np.float64).copy())
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


# ------------------------------------------------------------ chunk work --

_handles: dict = {}


def _chunk_handle(chunk, L: int):
    """A library handle of L qubits (no virtual chunks) attached to the
    chunk, on the chunk's device and current stream (cached per chunk)."""
    import ctypes
    import torch
    from . import sv
    key = (chunk.data_ptr(), L, chunk.dtype)
    h = _handles.get(key)
    if h is None:
        dt = sv.C64 if chunk.dtype == torch.complex64 else sv.C128
        h = sv._H()
        with torch.cuda.device(chunk.device):
            sv._check(sv._lib.sv_create(L, 0, dt, ctypes.byref(h)))
            sv._check(sv._lib.sv_attach_state(h, ctypes.c_void_p(chunk.data_ptr()),
                                              chunk.numel() * chunk.element_size()))
        _handles[key] = h
    sv._check(sv._lib.sv_set_stream(h, ctypes.c_void_p(torch.cuda.current_stream(chunk.device).cuda_stream)))
    return h


def release_handles() -> None:
    """Destroy the cached chunk handles (their chunks are not freed)."""
    from . import sv
    for h in _handles.values():
        sv._lib.sv_destroy(h)
    _handles.clear()


def local_circuit(circ, gate_ids, l2p) -> W.Circuit:
    """The tile's gates (in schedule order) with their targets as physical
    bits of the tile's layout; parameter and matrix indices unchanged."""
    ids = np.asarray(gate_ids, np.int64)
    q = circ.qubits[ids].copy()
    lp = np.asarray(l2p, np.int32)
    q[q >= 0] = lp[q[q >= 0]]
    return W.Circuit(circ.n, circ.kinds[ids].copy(), q, circ.param[ids].copy(), circ.mat[ids].copy(),
                     circ.nparams, circ.mats)


def apply_local(chunk, L: int, circ, params, gate_ids, l2p) -> None:
    """The tile's gates on one chunk: the gates' physical targets are all
    local (a tile of the lazy plan), so the chunk evolves as an L-qubit state
    under the library's kernels (one tile, no QR)."""
    import ctypes
    from . import sv
    if len(gate_ids) == 0:
        return
    c = local_circuit(circ, gate_ids, l2p)
    c.n = L
    h = _chunk_handle(chunk, L)
    gates = sv.gate_array(c)
    p = np.ascontiguousarray(params, np.float64)
    mats, nm = sv._mats(c)
    sv._check(sv._lib.sv_apply_circuit(h, sv._ptr(gates), c.m, sv._ptr(p), p.size,
                                       sv._ptr(mats) if mats is not None else None, nm, sv.DIRECT, None))


def expect_local(chunk, L: int, x, z):
    """Per string sum over the chunk of conj(psi[y ^ x]) i^nY (-1)^{y.z} psi[y]
    (x, z: physical masks on the local bits), by the library's EVC kernels
    with no device allocation, 256 strings per call."""
    from . import sv
    import torch
    dt = sv.C64 if chunk.dtype == torch.complex64 else sv.C128
    out = np.zeros(len(x), np.float64)
    for s in range(0, len(x), 256):
        p = sv.pauli_array(x[s:s + 256], z[s:s + 256])
        _, pt = sv.expect_noalloc(chunk, L, dt, p, np.ones(len(p)))
        out[s:s + 256] = pt
    return out


# ----------------------------------------------------------- orchestration --

def _physical(mask: int, l2p) -> int:
    out = 0
    q = 0
    while mask:
        if mask & 1:
            out |= 1 << int(l2p[q])
        mask >>= 1
        q += 1
    return out


def sharded_energy(n: int, circ, params, ham, chunk, init_index: int = 0, group=None, schedule=None,
                   options=None):
    """E = sum_t a_t <psi|P_t|psi> with psi = U|init> on the state sharded
    over the ranks of `group` (a power of two, 2^g ranks: global qubits = the
    top g physical bits).  QSU follows the library's plan under `schedule`
    (default the lazy plan, Alg. 1-3; the hierarchical plan, Alg. 4/5, with
    options.intra_bits global qubits inside a node): before each tile its QR
    (qr_exchange), then the tile's gates on every chunk; EVC follows the lazy
    EVC plan (Alg. 6, diagonalized targets) from the final QSU layout: per
    tile its QR, then every string's local sum, signed by the chunk's global
    bits under its Z letters; the per-string values are summed over the
    ranks.  `chunk` (2^L amplitudes) is overwritten.  Returns (energy,
    per-string values, final layout)."""
    import torch.distributed as dist
    from . import sv
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    g = world.bit_length() - 1
    if 1 << g != world:
        raise ValueError("sharded_energy: the number of ranks must be a power of two")
    L = n - g
    if chunk.numel() != 1 << L:
        raise ValueError("sharded_energy: the chunk must hold 2^(n - g) amplitudes")
    chunk.zero_()
    if init_index >> L == rank:
        chunk[init_index & ((1 << L) - 1)] = 1
    plan = sv.plan_qsu(n, g, circ, sv.LAZY if schedule is None else schedule, options)
    l2p = list(range(n))
    for t in plan["tiles"]:
        qr_exchange(chunk, L, rank, t["pairs"], group)
        apply_local(chunk, L, circ, params, plan["order"][t["begin"]:t["end"]], t["l2p"])
        l2p = t["l2p"]
    x, z = W.pauli_masks(ham)
    evc = sv.plan_evc(n, g, x, z, sv.LAZY, l2p=l2p)
    vals = np.zeros(len(x), np.float64)
    low = (1 << L) - 1
    for t in evc["tiles"]:
        qr_exchange(chunk, L, rank, t["pairs"], group)
        terms = evc["order"][t["begin"]:t["end"]]
        px = [_physical(int(x[i]), t["l2p"]) for i in terms]
        pz = [_physical(int(z[i]), t["l2p"]) for i in terms]
        if any(v >> L for v in px):
            raise NotImplementedError("sharded_energy: a string with X/Y on more qubits than a chunk holds")
        sign = np.array([-1.0 if bin((rank << L) & v).count("1") & 1 else 1.0 for v in pz])
        loc = expect_local(chunk, L, np.array(px, np.uint64), np.array([v & low for v in pz], np.uint64))
        vals[np.asarray(terms, np.int64)] = sign * loc
        l2p = t["l2p"]
    vals = allreduce_sum(vals, group, chunk.device if dist.get_backend(group) == "nccl" else None)
    return float(np.dot(ham.coeffs, vals)), vals, l2p


# ----------------------------------------------------------- cost model --

def qr_kinds(plan: dict, n: int) -> list[str]:
    """Per QR of a plan (sv.plan_qsu / plan_evc dict), 'intra' or 'inter'
    (Fig. 7): a QR is an inter QR when the inter set Q \\ (Q_L u Q_intra)
    changes, i.e. amplitudes cross nodes; otherwise they stay in a node."""
    full = (1 << n) - 1
    kinds, prev = [], None
    for t in plan["tiles"]:
        inter = full & ~(t["local_mask"] | t.get("intra_mask", 0))
        if t["pairs"]:
            kinds.append("inter" if prev is None or inter != prev else "intra")
        prev = inter
    return kinds


def qr_weight(n: int, g: int, s: int, amp_bytes: int, bandwidth_gbs: float) -> float:
    """Seconds of one QR of s pairs on 2^g ranks: every rank sends (and
    receives) 1 - 2^-s of its chunk of 2^(n - g) amplitudes over a link of
    the given bandwidth."""
    return (1.0 - 2.0 ** -s) * (1 << (n - g)) * amp_bytes / (bandwidth_gbs * 1e9)


def comm_cost(plan: dict, n: int, w_intra: float, w_inter: float) -> float:
    """Eq. comm_cost: w_intra * N_intra + w_inter * N_inter over the plan's QRs."""
    k = qr_kinds(plan, n)
    return w_intra * k.count("intra") + w_inter * k.count("inter")
