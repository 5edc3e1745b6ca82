"""Pins for the oracle planner (oracle/planner.py): the paper's worked
examples (Fig. 8 and Fig. 9 captions), brute-force checks and invariants."""
from itertools import combinations

import pytest

from conftest import read_golden
from oracle import planner as P
from paper_2410_04252_gb300 import workloads as W


def _sets(s):
    return [set(int(v) for v in part.split(",")) for part in s.split("|")]


def _tile_starts(plan):
    out, s = [], 0
    for t in plan.tiles:
        out.append(s)
        s += len(t)
    return out


def test_fig8_flat_tiling_caption():
    g = read_golden("fig8_flat_tiling.txt")
    n, nL = int(g["n"]), int(g["n_local"])
    c = W.fabric_blocks_circuit(n, int(g["layers"]))
    assert c.m == 42
    T = [c.targets(i) for i in range(c.m)]
    plan = P.flat_tiling(n, T, nL, pad="highest")
    starts = _tile_starts(plan)
    qr_after = [int(v) for v in g["qr_after_gate"].split()]
    for a in qr_after:
        assert a + 1 in starts
    assert plan.nqr == int(g["total_qrs"])
    gsets = [set(range(n)) - set(L) for L in plan.locals_]
    assert gsets[:3] == _sets(g["global_sets"])


def test_fig9_hierarchical_tiling_caption():
    g = read_golden("fig9_hierarchical_tiling.txt")
    n, nL, ni = int(g["n"]), int(g["n_local"]), int(g["n_intra"])
    c = W.fabric_blocks_circuit(n, int(g["layers"]))
    T = [c.targets(i) for i in range(c.m)]
    plan = P.hierarchical_tiling(n, T, nL, ni, pad="highest")
    assert _tile_starts(plan) == [int(v) for v in g["first_gate_of_tile"].split()]
    assert P.classify_hierarchical(plan, n) == g["qr_kinds"].split()
    assert [set(s) for s in plan.intra] == _sets(g["intra_sets"])
    inter = [set(range(n)) - set(L) - set(I) for L, I in zip(plan.locals_, plan.intra)]
    assert inter == _sets(g["inter_sets"])


def test_lowest_padding_contradicts_fig9():
    """The printed 'lowest qubit' padding does not give the caption's sets."""
    g = read_golden("fig9_hierarchical_tiling.txt")
    c = W.fabric_blocks_circuit(16, 12)
    T = [c.targets(i) for i in range(c.m)]
    plan = P.hierarchical_tiling(16, T, 12, 2, pad="lowest")
    assert [set(s) for s in plan.intra] != _sets(g["intra_sets"])


def test_depth_is_longest_path():
    """depth = longest chain of gates sharing qubits ending at the gate,
    computed here over all earlier gates, not just the last one per qubit."""
    for seed in range(5):
        c = W.random_circuit(7, 60, seed)
        T = [c.targets(i) for i in range(c.m)]
        d = P.depths(T)
        for j in range(c.m):
            best = 0
            for i in range(j):
                if set(T[i]) & set(T[j]):
                    best = max(best, d[i] + 1)
            assert d[j] == best


def check_qsu_plan(plan, T, n, nL, initial_identity=True):
    m = len(T)
    assert sorted(plan.order) == list(range(m))                 # each gate once
    pos = {u: i for i, u in enumerate(plan.order)}
    for j in range(m):                                          # C1
        for i in range(j):
            if set(T[i]) & set(T[j]):
                assert pos[i] < pos[j]
    l2p = list(range(n))
    cur = set(range(nL))
    for k, tile in enumerate(plan.tiles):
        assert tile                                             # non-empty
        for a, b in plan.qrs[k]:                                # apply the QR
            assert a < nL <= b
            la, lb = l2p.index(a), l2p.index(b)
            l2p[la], l2p[lb] = b, a
        assert l2p == plan.perms[k]
        assert sorted(l2p) == list(range(n))                    # bijection
        locs = {q for q in range(n) if l2p[q] < nL}
        assert locs == set(plan.locals_[k])
        for u in tile:                                          # C2
            assert set(T[u]) <= locs
        if k > 0:
            assert plan.locals_[k] != plan.locals_[k - 1]
            assert plan.qrs[k]
        cur = locs
    return cur


@pytest.mark.parametrize("pad", ["highest", "lowest"])
def test_flat_tiling_invariants(pad):
    for seed in range(12):
        n = 8 + seed % 5
        nL = n - 1 - seed % 3
        c = W.random_circuit(n, 80, 100 + seed)
        T = [c.targets(i) for i in range(c.m)]
        plan = P.flat_tiling(n, T, nL, pad)
        check_qsu_plan(plan, T, n, nL)
        # t tiles -> t - 1 QRs when the first tile keeps the initial mapping
        if plan.locals_[0] == frozenset(range(nL)):
            assert plan.nqr == len(plan.tiles) - 1


def test_flat_tiling_on_paper_workloads():
    for n, g, layers, ansatz in [(26, 4, 8, "fabric"), (30, 6, 12, "fabric"), (32, 6, 6, "hea"),
                                 (12, 2, 4, "hea")]:
        c = W.fabric_circuit(n, layers) if ansatz == "fabric" else W.hea_circuit(n, layers)
        T = [c.targets(i) for i in range(c.m)]
        plan = P.flat_tiling(n, T, n - g)
        check_qsu_plan(plan, T, n, n - g)
        ad = P.adhoc_schedule(n, T, n - g)
        check_qsu_plan(ad, T, n, n - g)
        assert plan.nqr <= ad.nqr


def test_adhoc_rule_definition():
    """Each QR of the ad hoc rule brings in exactly the global targets of the
    operation that triggers it, and evicts least recently used locals."""
    for seed in range(8):
        n, nL = 9, 6
        c = W.random_circuit(n, 60, 300 + seed)
        T = [c.targets(i) for i in range(c.m)]
        plan = P.adhoc_schedule(n, T, nL)
        check_qsu_plan(plan, T, n, nL)
        prev = set(range(nL))
        for k, tile in enumerate(plan.tiles):
            first = set(T[tile[0]])
            if plan.qrs[k]:
                assert set(plan.locals_[k]) - prev == first - prev
                assert len(plan.qrs[k]) == len(first - prev)
            prev = set(plan.locals_[k])


def test_qr_pairs_swap_by_physical_position():
    l2p = [3, 0, 5, 1, 2, 4]      # logical -> physical, nL = 3 (physical 0..2 local)
    old = {1, 3, 4}               # logical locals (phys 0, 1, 2)
    new = {1, 0, 5}
    pairs, after = P.qr_pairs(l2p, old, new)
    # outgoing: logical 3 (phys 1), 4 (phys 2); incoming: 0 (phys 3), 5 (phys 4)
    assert pairs == [(1, 3), (2, 4)]
    assert after == [1, 0, 5, 3, 4, 2]


def _greedy_check(n, nG, xmasks, plan):
    remaining = list(range(len(xmasks)))
    for tile, locs in zip(plan.tiles, plan.locals_):
        # brute force over local sets (not global sets) for the largest tile
        best = 0
        for L in combinations(range(n), n - nG):
            lm = sum(1 << q for q in L)
            cnt = sum(1 for i in remaining if xmasks[i] & ~lm == 0)
            best = max(best, cnt)
        assert len(tile) == best
        lm = sum(1 << q for q in locs)
        assert all(xmasks[i] & ~lm == 0 for i in tile)
        remaining = [i for i in remaining if i not in set(tile)]
    assert not remaining


@pytest.mark.parametrize("n,nG,kind", [(8, 2, "random"), (9, 3, "jw"), (10, 2, "random"),
                                       (10, 3, "jw")])
def test_alg6_greedy_and_diagonalized(n, nG, kind):
    h = W.random_hamiltonian(n, 60, 7 + n) if kind == "random" else W.jw_hamiltonian(n, 80, 9 + n)
    x, z = W.pauli_masks(h)
    xm = [int(v) for v in x]
    ok = [i for i in range(len(xm)) if bin(xm[i]).count("1") <= n - nG]
    xm = [xm[i] for i in ok]
    plan = P.tiling_pauli_strings(n, nG, xm)
    _greedy_check(n, nG, xm, plan)
    assert sorted(plan.order) == list(range(len(xm)))
    # strings without X/Y (pure Z / identity) fit every tile: all in the first
    for i, v in enumerate(xm):
        if v == 0:
            assert i in plan.tiles[0]


def test_evc_adhoc_index_order():
    n, nG = 9, 2
    h = W.random_hamiltonian(n, 50, 4)
    x, z = W.pauli_masks(h)
    plan = P.evc_adhoc(n, nG, x, z)
    assert plan.order == list(range(h.nterms))
    T = P.eager_evc_targets(n, n - nG, x, z)
    for tile, L in zip(plan.tiles, plan.locals_):
        for i in tile:
            assert set(T[i]) <= set(L)
