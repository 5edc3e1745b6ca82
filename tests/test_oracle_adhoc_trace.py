"""Pins the ad hoc (eager) QR rule of the oracle planner (the comparator of
Sec. V-B-1) to a trace worked out by hand in tests/golden, and shows that
the trace tells the reading apart from its plausible alternatives: each
alternative is planted in the oracle here, on the CPU, and must break the
trace.  The library planner must give the same trace (eager EVC plan of
Z strings whose supports are the operations' targets)."""
import pytest

from oracle import planner as P

from conftest import read_golden


def _golden():
    g = read_golden("adhoc_eviction_trace.txt")
    ops = [tuple(int(v) for v in s.split(",")) for s in g["ops"].split("|")]
    tile_ops = [[int(v) for v in s.split(",")] for s in g["tile_ops"].split("|")]
    tile_qrs = []
    for s in g["tile_qrs"].split("|"):
        s = s.strip()
        tile_qrs.append([tuple(int(v) for v in p.split("-")) for p in s.split(",")] if s else [])
    layouts = [[int(v) for v in s.split(",")] for s in g["tile_layouts"].split("|")]
    locals_ = [frozenset(int(v) for v in s.split(",")) for s in g["tile_locals"].split("|")]
    return int(g["n"]), int(g["n_local"]), ops, tile_ops, tile_qrs, layouts, locals_, int(g["total_qrs"])


def _trace(plan):
    return plan.tiles, [list(q) for q in plan.qrs], plan.perms, plan.locals_, plan.nqr


def test_adhoc_rule_matches_hand_trace():
    n, nL, ops, tile_ops, tile_qrs, layouts, locals_, nqr = _golden()
    plan = P.adhoc_schedule(n, ops, nL, order=list(range(len(ops))))
    tiles, qrs, perms, locs, count = _trace(plan)
    assert tiles == tile_ops
    assert qrs == tile_qrs
    assert perms == layouts
    assert locs == locals_
    assert count == nqr


_MUTANTS = {
    "most_recently_used": lambda cand, last: sorted(cand, key=lambda q: (-last[q], -q)),
    "ties_to_lowest": lambda cand, last: sorted(cand, key=lambda q: (last[q], q)),
    "never_used_last": lambda cand, last: sorted(cand, key=lambda q: (last[q] if last[q] >= 0 else 1 << 30, -q)),
}


@pytest.mark.parametrize("mutant", sorted(_MUTANTS))
def test_alternative_eviction_breaks_trace(mutant, monkeypatch):
    n, nL, ops, tile_ops, tile_qrs, layouts, locals_, nqr = _golden()
    monkeypatch.setattr(P, "adhoc_evict_order", _MUTANTS[mutant])
    plan = P.adhoc_schedule(n, ops, nL, order=list(range(len(ops))))
    assert (plan.qrs, plan.perms) != (tile_qrs, layouts)


def test_pairing_by_logical_index_breaks_trace(monkeypatch):
    n, nL, ops, tile_ops, tile_qrs, layouts, locals_, nqr = _golden()

    def by_logical(l2p, old_locals, new_locals):
        out, inn = sorted(old_locals - new_locals), sorted(new_locals - old_locals)
        new, pairs = list(l2p), []
        for a, b in zip(out, inn):
            pairs.append((l2p[a], l2p[b]))
            new[a], new[b] = l2p[b], l2p[a]
        return pairs, new

    monkeypatch.setattr(P, "qr_pairs", by_logical)
    plan = P.adhoc_schedule(n, ops, nL, order=list(range(len(ops))))
    assert (plan.qrs, plan.perms) != (tile_qrs, layouts)


def test_library_eager_evc_plan_matches_hand_trace():
    sv = pytest.importorskip("paper_2410_04252_gb300.sv")
    import numpy as np
    n, nL, ops, tile_ops, tile_qrs, layouts, locals_, nqr = _golden()
    # Z strings: no X/Y letters, full support = the operation's targets
    x = np.zeros(len(ops), dtype=np.uint64)
    z = np.array([sum(1 << q for q in t) for t in ops], dtype=np.uint64)
    lib = sv.plan_evc(n, n - nL, x, z, sv.EAGER)
    tiles = [lib["order"][t["begin"]:t["end"]] for t in lib["tiles"]]
    assert tiles == tile_ops
    assert [[tuple(p) for p in t["pairs"]] for t in lib["tiles"]] == tile_qrs
    assert [t["l2p"] for t in lib["tiles"]] == layouts


def _wide_golden():
    g = read_golden("wide_string_plan.txt")

    def mask(s):
        s = s.strip()
        return 0 if s == "-" else sum(1 << int(v) for v in s.split(","))

    def lists(s):
        return [[int(v) for v in t.split(",")] for t in s.split("|")]

    def qrs(s):
        out = []
        for t in s.split("|"):
            t = t.strip()
            out.append([] if t == "-" else [tuple(int(v) for v in p.split("-")) for p in t.split(",")])
        return out

    x = [mask(s) for s in g["x"].split("|")]
    z = [mask(s) for s in g["z"].split("|")]
    return (int(g["n"]), int(g["n_global"]), x, z,
            {k: (lists(g[k + "_tiles"]), qrs(g[k + "_qrs"]), lists(g[k + "_layouts"])) for k in ("lazy", "eager")})


def test_wide_string_tile_hand_plan():
    n, nG, x, z, want = _wide_golden()
    lazy = P.tiling_pauli_strings(n, nG, x)
    assert (lazy.tiles, [list(q) for q in lazy.qrs], lazy.perms) == want["lazy"]
    eager = P.evc_adhoc(n, nG, x, z)
    assert (eager.tiles, [list(q) for q in eager.qrs], eager.perms) == want["eager"]
    sv = pytest.importorskip("paper_2410_04252_gb300.sv")
    import numpy as np
    xa, za = np.array(x, dtype=np.uint64), np.array(z, dtype=np.uint64)
    for sched, key in ((sv.LAZY, "lazy"), (sv.EAGER, "eager")):
        lib = sv.plan_evc(n, nG, xa, za, sched)
        tiles = [lib["order"][t["begin"]:t["end"]] for t in lib["tiles"]]
        got = (tiles, [[tuple(p) for p in t["pairs"]] for t in lib["tiles"]], [t["l2p"] for t in lib["tiles"]])
        assert got == want[key]
