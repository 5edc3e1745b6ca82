"""Seeded synthetic inputs: circuits, parameters and Pauli Hamiltonians.

This module is shared by the CUDA path, its tests, the benchmark and the CPU
oracle.  It holds no arithmetic of the simulated method: it only draws random
numbers and lays out gate lists and Pauli strings.  Everything here stands in
for the paper's workloads (the GateFabric ansatz of Sec. V-A and the H2O
Jordan-Wigner Hamiltonians built with OpenFermion), whose data is not
available: circuits keep the paper's brick structure, Hamiltonians keep the
Jordan-Wigner shape (pure-Z terms plus X/Y pairs joined by a Z chain).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014):
    uniform u = (x >> 11) * 2**-53,
    normal via Box-Muller on two uniforms,
    Pauli letter = floor(4u) -> I, X, Y, Z.
Seeds: parameters 1000 + config, Hamiltonian 2000 + config, batched state i
3000 + i.

Gate kinds (integers shared with the C ABI): RY=0, RZ=1, CZ=2, GIVENS=3,
DEXC=4, MAT1=5, MAT2=6, MAT4=7.  A gate is (kind, qubits (up to 4, -1 pad),
parameter index or -1, matrix index or -1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RY, RZ, CZ, GIVENS, DEXC, MAT1, MAT2, MAT4 = range(8)
GATE_NQ = {RY: 1, RZ: 1, CZ: 2, GIVENS: 2, DEXC: 4, MAT1: 1, MAT2: 2, MAT4: 4}
GATE_NAMES = {RY: "RY", RZ: "RZ", CZ: "CZ", GIVENS: "GIVENS", DEXC: "DEXC",
              MAT1: "MAT1", MAT2: "MAT2", MAT4: "MAT4"}

# Pauli letter codes, one byte per qubit.
PI, PX, PY, PZ = 0, 1, 2, 3

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, one output per step)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self, sd: float = 1.0) -> float:
        u1 = self.uniform()
        u2 = self.uniform()
        return sd * math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)

    def randint(self, hi: int) -> int:
        """Integer in [0, hi)."""
        return min(int(self.uniform() * hi), hi - 1)


@dataclass
class Circuit:
    n: int
    kinds: np.ndarray          # int32 [m]
    qubits: np.ndarray         # int32 [m, 4], -1 padded
    param: np.ndarray          # int32 [m], -1 if none
    mat: np.ndarray            # int32 [m], -1 if none
    nparams: int
    mats: np.ndarray = field(default_factory=lambda: np.zeros((0,), np.float64))

    @property
    def m(self) -> int:
        return int(self.kinds.shape[0])

    def targets(self, i: int) -> tuple:
        return tuple(int(q) for q in self.qubits[i] if q >= 0)


@dataclass
class Hamiltonian:
    n: int
    letters: np.ndarray        # uint8 [nterms, n]: 0=I 1=X 2=Y 3=Z, qubit q in column q
    coeffs: np.ndarray         # float64 [nterms]

    @property
    def nterms(self) -> int:
        return int(self.coeffs.shape[0])


def _circuit(n, gates, nparams, mats=None):
    m = len(gates)
    kinds = np.zeros(m, np.int32)
    qubits = np.full((m, 4), -1, np.int32)
    param = np.full(m, -1, np.int32)
    mat = np.full(m, -1, np.int32)
    for i, (k, qs, p, mi) in enumerate(gates):
        kinds[i] = k
        qubits[i, :len(qs)] = qs
        param[i] = p
        mat[i] = mi
    return Circuit(n, kinds, qubits, param, mat, nparams,
                   np.zeros((0,), np.float64) if mats is None else np.asarray(mats, np.float64))


def hea_circuit(n: int, layers: int) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta_q) RZ(phi_q) on every
    qubit (listed qubit by qubit), then CZ(q, q+1) for q = 0..n-2.
    Layer l uses parameters theta_q = 2nl + q and phi_q = 2nl + n + q."""
    gates = []
    for l in range(layers):
        for q in range(n):
            gates.append((RY, (q,), 2 * n * l + q, -1))
            gates.append((RZ, (q,), 2 * n * l + n + q, -1))
        for q in range(n - 1):
            gates.append((CZ, (q, q + 1), -1, -1))
    return _circuit(n, gates, 2 * n * layers)


def fabric_circuit(n: int, layers: int) -> Circuit:
    """Particle-conserving brick ansatz shaped like GateFabric (Sec. V-A):
    layer l has offset 0 (l even) or 2 (l odd) and a 4-qubit block at every
    q = offset + 4j with q + 3 < n.  A block is DEXC(theta) on (q..q+3), then
    GIVENS(phi) on (q, q+2) and on (q+1, q+3); both Givens share phi.
    Block b uses parameters theta = 2b, phi = 2b + 1."""
    gates = []
    b = 0
    for l in range(layers):
        off = 0 if l % 2 == 0 else 2
        q = off
        while q + 3 < n:
            gates.append((DEXC, (q, q + 1, q + 2, q + 3), 2 * b, -1))
            gates.append((GIVENS, (q, q + 2), 2 * b + 1, -1))
            gates.append((GIVENS, (q + 1, q + 3), 2 * b + 1, -1))
            b += 1
            q += 4
    return _circuit(n, gates, 2 * b)


def fabric_blocks_circuit(n: int, layers: int) -> Circuit:
    """The same brick pattern with each 4-qubit block kept as ONE operator
    (a MAT4 slot without a matrix), as drawn in the paper's Fig. 8/9 for the
    16-qubit GateFabric example.  Used for planning only."""
    gates = []
    for l in range(layers):
        off = 0 if l % 2 == 0 else 2
        q = off
        while q + 3 < n:
            gates.append((MAT4, (q, q + 1, q + 2, q + 3), -1, -1))
            q += 4
    return _circuit(n, gates, 0)


def uniform_params(count: int, seed: int, lo: float, hi: float) -> np.ndarray:
    rng = SplitMix64(seed)
    return np.array([lo + (hi - lo) * rng.uniform() for _ in range(count)], np.float64)


def random_hamiltonian(n: int, nterms: int, seed: int) -> Hamiltonian:
    """Each qubit of each string is I/X/Y/Z with probability 1/4; the
    coefficient is drawn after the letters, N(0, 1)."""
    rng = SplitMix64(seed)
    letters = np.zeros((nterms, n), np.uint8)
    coeffs = np.zeros(nterms, np.float64)
    for t in range(nterms):
        for q in range(n):
            letters[t, q] = min(int(4.0 * rng.uniform()), 3)
        coeffs[t] = rng.normal(1.0)
    return Hamiltonian(n, letters, coeffs)


def _distinct_pair(rng: SplitMix64, n: int):
    i = rng.randint(n)
    j = rng.randint(n - 1)
    if j >= i:
        j += 1
    return (i, j) if i < j else (j, i)


def jw_hamiltonian(n: int, nterms: int, seed: int) -> Hamiltonian:
    """Jordan-Wigner-shaped strings.  The first quarter are pure-Z terms
    (first half of those weight 1, second half weight 2 on distinct random
    qubits) with N(0, 1) coefficients; the rest are X/Y pairs on a random
    i < j, each endpoint X or Y with probability 1/2, Z on every qubit
    strictly between, with N(0, 0.1) coefficients (0.1 = standard deviation)."""
    rng = SplitMix64(seed)
    letters = np.zeros((nterms, n), np.uint8)
    coeffs = np.zeros(nterms, np.float64)
    nz = nterms // 4
    for t in range(nterms):
        if t < nz:
            if t < nz // 2:
                letters[t, rng.randint(n)] = PZ
            else:
                i, j = _distinct_pair(rng, n)
                letters[t, i] = PZ
                letters[t, j] = PZ
            coeffs[t] = rng.normal(1.0)
        else:
            i, j = _distinct_pair(rng, n)
            letters[t, i] = PX if rng.uniform() < 0.5 else PY
            letters[t, j] = PX if rng.uniform() < 0.5 else PY
            for q in range(i + 1, j):
                letters[t, q] = PZ
            coeffs[t] = rng.normal(0.1)
    return Hamiltonian(n, letters, coeffs)


def pauli_masks(h: Hamiltonian):
    """(x, z) bit masks per string: x has the X/Y positions, z the Z/Y
    positions (Y = both).  Pure relabelling of the letters."""
    x = np.zeros(h.nterms, np.uint64)
    z = np.zeros(h.nterms, np.uint64)
    for t in range(h.nterms):
        xv = 0
        zv = 0
        for q in range(h.n):
            c = int(h.letters[t, q])
            if c in (PX, PY):
                xv |= 1 << q
            if c in (PZ, PY):
                zv |= 1 << q
        x[t] = xv
        z[t] = zv
    return x, z


def half_filled_index(n: int) -> int:
    """Basis state with the lowest n/2 qubits set."""
    return (1 << (n // 2)) - 1


# The five workloads.  'n_small' is the oracle-sized copy used for parity at
# full-size structure (same generators, smaller n).
CONFIGS = {
    0: dict(name="hea_n12_g2_c128", n=12, g=2, dtype="c128", ansatz="hea", layers=4,
            ham="random", nterms=64, schedule="eager", init=0,
            param_lo=0.0, param_hi=2.0 * math.pi, work="qsu+evc"),
    1: dict(name="fabric_n26_g4_c64", n=26, g=4, dtype="c64", ansatz="fabric", layers=8,
            ham=None, nterms=0, schedule="lazy", init="half",
            param_lo=-math.pi, param_hi=math.pi, work="qsu"),
    2: dict(name="fabric_n30_g6_c64_jw4096", n=30, g=6, dtype="c64", ansatz="fabric", layers=12,
            ham="jw", nterms=4096, schedule="lazy", init="half",
            param_lo=-math.pi, param_hi=math.pi, work="qsu+evc", n_small=20),
    3: dict(name="hea_n32_g6_c64_rand1024_adjoint", n=32, g=6, dtype="c64", ansatz="hea", layers=6,
            ham="random", nterms=1024, schedule="lazy", init=0,
            param_lo=0.0, param_hi=2.0 * math.pi, work="qsu+evc+grad", n_small=14),
    4: dict(name="batch256_hea_n18_c64_rand512", n=18, g=0, dtype="c64", ansatz="hea", layers=8,
            ham="random", nterms=512, schedule="lazy", init=0, batch=256, min_layers=2,
            param_lo=0.0, param_hi=2.0 * math.pi, work="batch"),
}


def make_circuit(cfg: dict, n: int | None = None, layers: int | None = None) -> Circuit:
    n = cfg["n"] if n is None else n
    layers = cfg["layers"] if layers is None else layers
    if cfg["ansatz"] == "hea":
        return hea_circuit(n, layers)
    return fabric_circuit(n, layers)


def make_params(cfg_id: int, circ: Circuit) -> np.ndarray:
    cfg = CONFIGS[cfg_id]
    return uniform_params(circ.nparams, 1000 + cfg_id, cfg["param_lo"], cfg["param_hi"])


def make_hamiltonian(cfg_id: int, n: int | None = None) -> Hamiltonian | None:
    cfg = CONFIGS[cfg_id]
    n = cfg["n"] if n is None else n
    if cfg["ham"] is None:
        return None
    if cfg["ham"] == "jw":
        return jw_hamiltonian(n, cfg["nterms"], 2000 + cfg_id)
    return random_hamiltonian(n, cfg["nterms"], 2000 + cfg_id)


def make_init(cfg: dict, n: int | None = None) -> int:
    n = cfg["n"] if n is None else n
    return half_filled_index(n) if cfg["init"] == "half" else int(cfg["init"])


def batch_states(count: int, n: int, max_layers: int, min_layers: int):
    """Per-state (layers, params) for the batched workload: state i draws
    its depth uniformly from [min_layers, max_layers] and then its
    parameters U[0, 2pi), all from seed 3000 + i."""
    out = []
    for i in range(count):
        rng = SplitMix64(3000 + i)
        layers = min_layers + rng.randint(max_layers - min_layers + 1)
        params = np.array([2.0 * math.pi * rng.uniform() for _ in range(2 * n * layers)], np.float64)
        out.append((layers, params))
    return out


def random_circuit(n: int, m: int, seed: int, kinds=(RY, RZ, CZ, GIVENS, DEXC)) -> Circuit:
    """Random gate list for property tests: each gate a random kind from
    `kinds` on random distinct qubits, each parametric gate with its own
    parameter."""
    rng = SplitMix64(seed)
    gates = []
    np_ = 0
    for _ in range(m):
        k = kinds[rng.randint(len(kinds))]
        nq = GATE_NQ[k]
        if nq > n:
            continue
        qs = []
        while len(qs) < nq:
            q = rng.randint(n)
            if q not in qs:
                qs.append(q)
        p = -1
        if k in (RY, RZ, GIVENS, DEXC):
            p = np_
            np_ += 1
        gates.append((k, tuple(qs), p, -1))
    return _circuit(n, gates, np_)


def random_unitary_mats(count: int, dim: int, seed: int) -> np.ndarray:
    """`count` Haar-like random unitaries of size dim x dim, interleaved
    (re, im) float64, via QR of a complex Gaussian matrix drawn from
    SplitMix64 normals."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        a = np.array([[complex(rng.normal(), rng.normal()) for _ in range(dim)] for _ in range(dim)])
        q, r = np.linalg.qr(a)
        d = np.diag(r)
        q = q * (d / np.abs(d))
        out.append(q)
    arr = np.stack(out) if out else np.zeros((0, dim, dim), complex)
    return np.ascontiguousarray(np.stack([arr.real, arr.imag], axis=-1)).reshape(-1)
