"""The library's host planner (C++) against the oracle planner (Python):
schedules, tile boundaries, QR pairs and layouts must be bit-exact.  Runs
without a GPU (planning makes no CUDA call)."""
import numpy as np
import pytest

from oracle import planner as P
from paper_2410_04252_gb300 import workloads as W

sv = pytest.importorskip("paper_2410_04252_gb300.sv")


def _same_qsu(lib, orc):
    assert lib["order"] == orc.order
    assert [t["pairs"] for t in lib["tiles"]] == [[tuple(p) for p in q] for q in orc.qrs]
    assert [t["l2p"] for t in lib["tiles"]] == orc.perms
    assert [t["local_mask"] for t in lib["tiles"]] == [sum(1 << q for q in L) for L in orc.locals_]
    starts = [t["begin"] for t in lib["tiles"]]
    ostarts, s = [], 0
    for t in orc.tiles:
        ostarts.append(s)
        s += len(t)
    assert starts == ostarts


@pytest.mark.parametrize("cfg", [0, 1, 2, 3])
@pytest.mark.parametrize("sched", ["lazy", "eager"])
def test_qsu_plan_configs(cfg, sched):
    cf = W.CONFIGS[cfg]
    circ = W.make_circuit(cf)
    n, nL = cf["n"], cf["n"] - cf["g"]
    T = [circ.targets(i) for i in range(circ.m)]
    lib = sv.plan_qsu(n, cf["g"], circ, sv.LAZY if sched == "lazy" else sv.EAGER)
    orc = P.flat_tiling(n, T, nL) if sched == "lazy" else P.adhoc_schedule(n, T, nL)
    _same_qsu(lib, orc)


@pytest.mark.parametrize("pad", ["highest", "lowest"])
def test_qsu_plan_random(pad):
    for seed in range(40):
        n = 6 + seed % 9
        g = 1 + seed % min(4, n - 4)
        c = W.random_circuit(n, 30 + 5 * (seed % 7), 500 + seed)
        T = [c.targets(i) for i in range(c.m)]
        rng = W.SplitMix64(900 + seed)
        l2p = list(range(n))
        if seed % 3 == 0:                     # a non-identity starting layout
            for i in range(n - 1, 0, -1):
                j = rng.randint(i + 1)
                l2p[i], l2p[j] = l2p[j], l2p[i]
        opt = sv.default_options()
        opt.pad_highest = 1 if pad == "highest" else 0
        lib = sv.plan_qsu(n, g, c, sv.LAZY, opt, l2p)
        _same_qsu(lib, P.flat_tiling(n, T, n - g, pad, l2p=l2p))
        lib = sv.plan_qsu(n, g, c, sv.EAGER, opt, l2p)
        _same_qsu(lib, P.adhoc_schedule(n, T, n - g, l2p=l2p))


def test_fig8_from_library_planner():
    c = W.fabric_blocks_circuit(16, 12)
    lib = sv.plan_qsu(16, 4, c, sv.LAZY)
    assert [t["begin"] for t in lib["tiles"]] == [0, 9, 24, 37]
    assert sum(1 for t in lib["tiles"] if t["pairs"]) == 3


def _same_evc(lib, orc):
    tiles = [lib["order"][t["begin"]:t["end"]] for t in lib["tiles"]]
    assert tiles == orc.tiles
    assert [t["pairs"] for t in lib["tiles"]] == [[tuple(p) for p in q] for q in orc.qrs]
    assert [t["l2p"] for t in lib["tiles"]] == orc.perms


@pytest.mark.parametrize("kind", ["random", "jw"])
def test_evc_plan_lazy_and_eager(kind):
    for seed in range(10):
        n = 7 + seed % 5
        g = 1 + seed % 3
        h = (W.random_hamiltonian(n, 40, 40 + seed) if kind == "random"
             else W.jw_hamiltonian(n, 64, 60 + seed))
        x, z = W.pauli_masks(h)          # includes strings wider than n_L
        rng = W.SplitMix64(70 + seed)
        l2p = list(range(n))
        if seed % 2:
            for i in range(n - 1, 0, -1):
                j = rng.randint(i + 1)
                l2p[i], l2p[j] = l2p[j], l2p[i]
        lib = sv.plan_evc(n, g, x, z, sv.LAZY, l2p=l2p)
        _same_evc(lib, P.tiling_pauli_strings(n, g, [int(v) for v in x], l2p=l2p))
        lib = sv.plan_evc(n, g, x, z, sv.EAGER, l2p=l2p)
        _same_evc(lib, P.evc_adhoc(n, g, x, z, l2p=l2p))


def test_gate_pass_invariants():
    """Each tile's gates are split into passes that stage the low bits, hold
    every target of their gates, apply each gate once, and keep C1."""
    for cfg in (1, 2, 3):
        cf = W.CONFIGS[cfg]
        circ = W.make_circuit(cf)
        for sched in (sv.LAZY, sv.EAGER):
            opt = sv.default_options()
            lib = sv.plan_qsu(cf["n"], cf["g"], circ, sched, opt)
            nL = cf["n"] - cf["g"]
            seen = []
            for ps in lib["passes"]:
                tile = lib["tiles"][ps["tile"]]
                bits = ps["bits"]
                assert bits & ((1 << opt.low_bits) - 1) == (1 << opt.low_bits) - 1
                assert bits < (1 << nL)
                assert bin(bits).count("1") <= opt.tile_bits
                for u in ps["ops"]:
                    assert u in lib["order"][tile["begin"]:tile["end"]]
                    for q in circ.targets(u):
                        assert bits >> tile["l2p"][q] & 1
                seen.extend(ps["ops"])
            assert sorted(seen) == list(range(circ.m))
            pos = {u: i for i, u in enumerate(seen)}
            T = [circ.targets(i) for i in range(circ.m)]
            last = {}
            for j in range(circ.m):
                for q in T[j]:
                    if q in last:
                        assert pos[last[q]] < pos[j]
                    last[q] = j


def test_invalid_inputs_rejected():
    c = W._circuit(4, [(W.RY, (0, 0), 0, -1)], 1)
    bad = W._circuit(4, [(W.CZ, (0, 0), -1, -1)], 0)
    with pytest.raises(sv.SvError) as e:
        sv.plan_qsu(4, 0, bad, sv.LAZY)
    assert e.value.status == sv.SV_EINVAL
    far = W._circuit(4, [(W.RY, (7,), 0, -1)], 1)
    with pytest.raises(sv.SvError):
        sv.plan_qsu(4, 0, far, sv.LAZY)
    # a string with more X/Y than local qubits: last tile, no QR
    p = sv.plan_evc(6, 2, [0b111111, 0b11], [0, 0], sv.LAZY)
    assert p["order"][-1] == 0 and not p["tiles"][-1]["pairs"]
    del c
