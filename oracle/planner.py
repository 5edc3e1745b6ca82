"""CPU ORACLE -- test infrastructure, not part of the product.

The paper's scheduling algorithms, written out step by step in the paper's
order and notation, independent of the library's C++ planner:

  depth / depth_sort        gate depth = critical-path length (Sec. III-A,
                            Fig. 1); stable sort by depth with ties broken by
                            the sorted target tuple, then input position
                            (Sec. IV-A-1, "prioritizes the target qubits in
                            ascending order")
  tile_construction         Alg. 2 (P1)
  qubit_mapping             Alg. 3 (P2), padding rule selectable
  flat_tiling               Alg. 1
  hierarchical_tiling       Alg. 4 with Alg. 5
  adhoc_schedule            the ad hoc (eager) scheduler of Sec. V-B-1: depth
                            order, and before each wide gate a new mapping
                            chosen for that gate alone (least recently used
                            local qubits are evicted, adhoc_evict_order; the
                            paper gives no rule, so this reading is pinned
                            by a trace worked out by hand from it, which
                            each alternative reading breaks)
  qr_pairs                  physical pairing of one QR (Sec. III-B-4: a
                            subset of Q_L exchanged with an equal-sized
                            subset of Q_G)
  tiling_pauli_strings      Alg. 6 with diagonalization (Eq. without_QR) and
                            merging of identical X/Y supports
  evc_adhoc                 index-order EVC with ad hoc QRs (Sec. V-B-2)

Readings taken where the paper is silent or inconsistent:
  * Alg. 1 removes the gate just scheduled (the printed loop increments x
    first).
  * Alg. 2 and Alg. 3 scan the depth-ordered list once; removing a gate does
    not shift the scan.
  * Alg. 3 pads with the HIGHEST free qubit by default: the captions of
    Fig. 8 and Fig. 9 are reproduced only that way; pad="lowest" is the
    printed text.
  * An empty first tile (first gate not narrow under the initial mapping) is
    dropped; the mapping change before the first gate then counts as a QR,
    as Eq. n_qr does with M(g(-1)) = {0..n_L-1}.
  * QR pairing: outgoing local qubits and incoming global qubits, each sorted
    by current physical position, are swapped pairwise.
  * Alg. 6 enumerates global sets as lexicographic combinations and keeps
    the first maximum (strict '<' in the paper's update).
  * Eager EVC uses a string's full support T(P) when it fits n_L qubits and
    its X/Y support otherwise (full support alone cannot make such strings
    narrow).
  * A string with more X/Y positions than local qubits fits no mapping (the
    paper does not treat this case); both EVC schedules put such strings in
    one last tile without a QR, whose amplitude pairs cross chunks.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations


# --------------------------------------------------------------------------
# Depth and ordering
# --------------------------------------------------------------------------

def depths(targets: list[tuple]) -> list[int]:
    """depth(U_i) = 0 if no earlier gate shares a qubit, else 1 + the largest
    depth among earlier gates sharing a qubit."""
    last = {}
    d = []
    for t in targets:
        di = 0
        for q in t:
            if q in last:
                di = max(di, last[q] + 1)
        for q in t:
            last[q] = di
        d.append(di)
    return d


def depth_sort(targets: list[tuple]) -> list[int]:
    d = depths(targets)
    return sorted(range(len(targets)), key=lambda i: (d[i], tuple(sorted(targets[i])), i))


# --------------------------------------------------------------------------
# Alg. 2 and Alg. 3
# --------------------------------------------------------------------------

def tile_construction(QL: set, remain: list[int], T: list[tuple]) -> list[int]:
    """Alg. 2: one pass in depth order; a gate joins the tile if its targets
    are all still available, otherwise its targets become unavailable."""
    avail = set(QL)
    G = []
    for u in remain:
        tu = set(T[u])
        if tu <= avail:
            G.append(u)
        else:
            avail -= tu
        if not avail:
            break
    return G


def qubit_mapping(Q: set, remain: list[int], T: list[tuple], nL: int, pad: str = "highest") -> set:
    """Alg. 3: union the targets of shallow remaining gates while they fit in
    nL qubits; a gate that cannot be taken blocks its targets.  Then pad."""
    avail = set(Q)
    QL = set()
    for u in remain:
        tu = set(T[u])
        if tu <= avail and len(QL | tu) <= nL:
            QL |= tu
        else:
            avail -= tu
        if not avail:
            break
    if not QL:
        return set()
    free = sorted(set(Q) - QL)
    while len(QL) < nL:
        q = free.pop() if pad == "highest" else free.pop(0)
        QL.add(q)
    return QL


# --------------------------------------------------------------------------
# Plans
# --------------------------------------------------------------------------

@dataclass
class Plan:
    n: int
    nL: int
    order: list = field(default_factory=list)        # schedule g: gate (or string) indices
    tiles: list = field(default_factory=list)        # list of lists of indices
    locals_: list = field(default_factory=list)      # per tile: frozenset of logical local qubits
    qrs: list = field(default_factory=list)          # per tile: list of (phys_local, phys_global) swapped before it
    perms: list = field(default_factory=list)        # per tile: logical->physical list in force for it
    intra: list = field(default_factory=list)        # hierarchical only: per tile Q_intra

    @property
    def nqr(self) -> int:
        return sum(1 for q in self.qrs if q)


def qr_pairs(l2p: list[int], old_locals: set, new_locals: set):
    """Physical pairs of one QR and the logical->physical map after it.
    Outgoing locals and incoming globals are each sorted by current physical
    position and swapped pairwise."""
    out = sorted(old_locals - new_locals, key=lambda q: l2p[q])
    inn = sorted(new_locals - old_locals, key=lambda q: l2p[q])
    assert len(out) == len(inn)
    new = list(l2p)
    pairs = []
    for a, b in zip(out, inn):
        pa, pb = l2p[a], l2p[b]
        pairs.append((pa, pb))
        new[a], new[b] = pb, pa
    return pairs, new


def _emit_tile(plan: Plan, tile, QL, l2p, cur_locals, intra=None):
    pairs = []
    if set(QL) != set(cur_locals):
        pairs, l2p = qr_pairs(l2p, set(cur_locals), set(QL))
    plan.tiles.append(list(tile))
    plan.order.extend(tile)
    plan.locals_.append(frozenset(QL))
    plan.qrs.append(pairs)
    plan.perms.append(list(l2p))
    if intra is not None:
        plan.intra.append(frozenset(intra))
    return l2p, set(QL)


def flat_tiling(n: int, T: list[tuple], nL: int, pad: str = "highest", l2p=None) -> Plan:
    """Alg. 1: alternate (P1) tile construction and (P2) remapping."""
    plan = Plan(n, nL)
    Q = set(range(n))
    l2p = list(range(n)) if l2p is None else list(l2p)
    cur = {q for q in range(n) if l2p[q] < nL}
    QL = set(cur)          # {0..n_L-1} for the identity layout (Alg. 1, line 2)
    remain = depth_sort(T)
    while remain:
        G = tile_construction(QL, remain, T)
        if G:
            l2p, cur = _emit_tile(plan, G, QL, l2p, cur)
            gs = set(G)
            remain = [u for u in remain if u not in gs]
        if not remain:
            break
        QL = qubit_mapping(Q, remain, T, nL, pad)
    return plan


def hierarchical_tiling(n: int, T: list[tuple], nL: int, nintra: int, pad: str = "highest") -> Plan:
    """Alg. 4 with Alg. 5 (two-phase remapping: an intra QR if the next local
    set can be drawn from Q_L and Q_intra, else an inter QR)."""
    plan = Plan(n, nL)
    Q = set(range(n))
    l2p = list(range(n))
    cur = set(range(nL))
    QL = set(range(nL))
    Qintra = set(range(nL, nL + nintra))
    remain = depth_sort(T)
    while remain:
        G = tile_construction(QL, remain, T)
        if G:
            l2p, cur = _emit_tile(plan, G, QL, l2p, cur, intra=Qintra)
            gs = set(G)
            remain = [u for u in remain if u not in gs]
        if not remain:
            break
        QLn = qubit_mapping(QL | Qintra, remain, T, len(QL), pad)
        if QLn:
            Qintra = (QL | Qintra) - QLn
        else:
            QLn = qubit_mapping(Q, remain, T, len(QL), pad)
            Qp = qubit_mapping(Q, remain, T, len(QL) + len(Qintra), pad)
            Qintra = Qp - QLn
        QL = QLn
    return plan


def classify_hierarchical(plan: Plan, n: int) -> list[str]:
    """Per tile transition: 'inter' if the inter set Q - (Q_L u Q_intra)
    changed, else 'intra' (Fig. 7's categorization)."""
    kinds = []
    for i in range(1, len(plan.tiles)):
        inter_old = set(range(n)) - plan.locals_[i - 1] - plan.intra[i - 1]
        inter_new = set(range(n)) - plan.locals_[i] - plan.intra[i]
        kinds.append("inter" if inter_old != inter_new else "intra")
    return kinds


def adhoc_evict_order(cand: set, last: list[int]) -> list[int]:
    """Eviction order of the ad hoc rule among candidate local qubits: least
    recently used first (last[q] = position of the last operation touching
    q, -1 if none), ties to the highest logical index."""
    return sorted(cand, key=lambda q: (last[q], -q))


def adhoc_schedule(n: int, T: list[tuple], nL: int, l2p=None, order=None) -> Plan:
    """Ad hoc (eager) QR: process in depth order (or the given order); before
    an operation whose targets are not all local, bring its global targets in
    by evicting the same number of locals outside its targets, least recently
    used first (never used counts as -1), ties to the highest logical index.
    A tile is a maximal run of operations under one mapping."""
    plan = Plan(n, nL)
    l2p = list(range(n)) if l2p is None else list(l2p)
    QL = {q for q in range(n) if l2p[q] < nL}
    last = [-1] * n
    seq = depth_sort(T) if order is None else list(order)
    tile = []
    pending = []          # pairs swapped before the tile being filled
    for x, u in enumerate(seq):
        tu = set(T[u])
        if not tu <= QL:
            inn = tu - QL
            cand = adhoc_evict_order(QL - tu, last)
            evict = set(cand[:len(inn)])
            newQL = (QL - evict) | inn
            pairs, l2p_new = qr_pairs(l2p, QL, newQL)
            if tile:
                plan.tiles.append(tile)
                plan.order.extend(tile)
                plan.locals_.append(frozenset(QL))
                plan.qrs.append(pending)
                plan.perms.append(list(l2p))
            tile = []
            pending = pairs
            l2p = l2p_new
            QL = newQL
        tile.append(u)
        for q in tu:
            last[q] = x
    if tile:
        plan.tiles.append(tile)
        plan.order.extend(tile)
        plan.locals_.append(frozenset(QL))
        plan.qrs.append(pending)
        plan.perms.append(list(l2p))
    return plan


# --------------------------------------------------------------------------
# EVC
# --------------------------------------------------------------------------

def x_support(xmask: int) -> frozenset:
    return frozenset(q for q in range(64) if (xmask >> q) & 1)


def tiling_pauli_strings(n: int, nG: int, xmasks: list[int], l2p=None) -> Plan:
    """Alg. 6 with diagonalization: a string's target for tiling is its X/Y
    support (Z on a global qubit becomes a per-chunk sign, Eq. par_exp).
    Strings with identical supports are merged, counted with multiplicity.
    Each step takes the first global set (lexicographic combinations) whose
    complement holds the most remaining strings.  Strings with more X/Y
    positions than local qubits fit no mapping; they form one last tile
    evaluated without a QR (see wide_tile)."""
    nL = n - nG
    plan = Plan(n, nL)
    l2p = list(range(n)) if l2p is None else list(l2p)
    cur = {q for q in range(n) if l2p[q] < nL}
    groups = {}
    wide = []
    for i, x in enumerate(xmasks):
        if bin(int(x)).count("1") > nL:
            wide.append(i)
            continue
        groups.setdefault(int(x), []).append(i)
    remaining = dict(groups)
    full = (1 << n) - 1
    while remaining:
        best = 0
        bestG = None
        for G in combinations(range(n), nG):
            gm = 0
            for q in G:
                gm |= 1 << q
            cnt = 0
            for x, members in remaining.items():
                if x & gm == 0:
                    cnt += len(members)
            if best < cnt:
                best = cnt
                bestG = gm
        take = sorted(x for x in remaining if x & bestG == 0)
        tile = sorted(i for x in take for i in remaining[x])
        for x in take:
            del remaining[x]
        QL = {q for q in range(n) if not (full & bestG) >> q & 1}
        l2p, cur = _emit_tile(plan, tile, QL, l2p, cur)
    wide_tile(plan, wide, l2p, cur)
    return plan


def wide_tile(plan: Plan, wide: list[int], l2p, cur) -> None:
    """Reading for strings whose X/Y support exceeds n_L (the paper's
    method has no mapping for them): one last tile, no QR, whose pairs
    (b, b ^ x) cross chunks."""
    if wide:
        plan.tiles.append(sorted(wide))
        plan.order.extend(sorted(wide))
        plan.locals_.append(frozenset(cur))
        plan.qrs.append([])
        plan.perms.append(list(l2p))


def eager_evc_targets(n: int, nL: int, xmasks, zmasks) -> list[tuple]:
    T = []
    for x, z in zip(xmasks, zmasks):
        full = int(x) | int(z)
        sup = [q for q in range(n) if (full >> q) & 1]
        if len(sup) > nL:
            sup = [q for q in range(n) if (int(x) >> q) & 1]
        T.append(tuple(sup))
    return T


def evc_adhoc(n: int, nG: int, xmasks, zmasks, l2p=None) -> Plan:
    """Index-order EVC with ad hoc QRs (the QSU-based baseline's order);
    strings wider than n_L go to one last tile without a QR."""
    nL = n - nG
    T = eager_evc_targets(n, nL, xmasks, zmasks)
    narrow = [i for i in range(len(T)) if len(T[i]) <= nL]
    wide = [i for i in range(len(T)) if len(T[i]) > nL]
    plan = adhoc_schedule(n, T, nL, l2p=l2p, order=narrow)
    last = plan.perms[-1] if plan.perms else (list(range(n)) if l2p is None else list(l2p))
    wide_tile(plan, wide, last, {q for q in range(n) if last[q] < nL})
    return plan
