"""ctypes binding of libsv (include/sv.h).  Argument marshalling only: every
step of the simulation runs in the library's CUDA kernels.  PyTorch provides
the device buffers (state, lambda) and the stream.

Importing this module fails loudly if the CUDA library has not been built;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsv.so not found at {LIB_PATH}: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_EPLAN, SV_ETIMEOUT, SV_EDEVICE, SV_ESTATE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EPLAN", "ETIMEOUT", "EDEVICE", "ESTATE"]
C64, C128 = 0, 1
EAGER, LAZY, DIRECT, HIER, LAZY_DIAG = 0, 1, 2, 3, 4
KEEP_LAYOUT, FORWARD_DONE = 1, 2


class SvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsv {STATUS_NAMES[status] if status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q", ctypes.c_int32 * 4), ("param", ctypes.c_int32),
                ("mat", ctypes.c_int32)]


class Pauli(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint64), ("z", ctypes.c_uint64)]


class Options(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("low_bits", ctypes.c_int32),
                ("evc_low_bits", ctypes.c_int32), ("evc_span", ctypes.c_int32),
                ("pad_highest", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("wait_limit", ctypes.c_int64), ("profile", ctypes.c_int32), ("fuse_max", ctypes.c_int32), ("intra_bits", ctypes.c_int32), ("plan_device", ctypes.c_int32)]


K_GATE, K_QR, K_EVC, K_HPSI, K_ADJ, K_PERM, K_AUX, K_BATCH = range(8)
KERNEL_KINDS = ["gate", "qr", "evc", "hpsi", "adj", "perm", "aux", "batch"]


class Stats(ctypes.Structure):
    _fields_ = [("qsu_tiles", ctypes.c_int32), ("qsu_qrs", ctypes.c_int32), ("qsu_passes", ctypes.c_int32),
                ("evc_tiles", ctypes.c_int32), ("evc_qrs", ctypes.c_int32), ("evc_passes", ctypes.c_int32),
                ("hpsi_passes", ctypes.c_int32), ("adj_passes", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("plan_cache_hit", ctypes.c_int32),
                ("plan_ms", ctypes.c_double),
                ("kernels", ctypes.c_int32 * 8),
                ("bytes", ctypes.c_double * 8), ("ms", ctypes.c_double * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("kernels", "bytes", "ms")}
        for i, k in enumerate(KERNEL_KINDS):
            d[f"kernels_{k}"] = self.kernels[i]
            d[f"bytes_{k}"] = self.bytes[i]
            d[f"ms_{k}"] = self.ms[i]
        return d


_vp, _sz, _i32, _u32, _u64, _dp = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.POINTER(ctypes.c_double))
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_H = ctypes.c_void_p

EXPORTS = {
    "sv_options_default": (None, [ctypes.c_int, ctypes.POINTER(Options)]),
    "sv_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_H)]),
    "sv_destroy": (None, [_H]),
    "sv_attach_state": (ctypes.c_int, [_H, _vp, _sz]),
    "sv_attach_buffer": (ctypes.c_int, [_H, _vp, _sz]),
    "sv_attach_lambda": (ctypes.c_int, [_H, _vp, _sz]),
    "sv_set_stream": (ctypes.c_int, [_H, _vp]),
    "sv_set_options": (ctypes.c_int, [_H, ctypes.POINTER(Options)]),
    "sv_get_options": (ctypes.c_int, [_H, ctypes.POINTER(Options)]),
    "sv_reset_basis": (ctypes.c_int, [_H, _u64]),
    "sv_set_state": (ctypes.c_int, [_H, _vp, ctypes.c_int]),
    "sv_get_state": (ctypes.c_int, [_H, _vp, ctypes.c_int, ctypes.c_int]),
    "sv_get_permutation": (ctypes.c_int, [_H, _i32p]),
    "sv_apply_circuit": (ctypes.c_int, [_H, _vp, _sz, _vp, _sz, _vp, _sz, ctypes.c_int, ctypes.POINTER(Stats)]),
    "sv_expect": (ctypes.c_int, [_H, _vp, _vp, _sz, ctypes.c_int, _u32, _dp, _vp, ctypes.POINTER(Stats)]),
    "sv_apply_hamiltonian": (ctypes.c_int, [_H, _vp, _vp, _sz, _vp, _dp, ctypes.POINTER(Stats)]),
    "sv_grad": (ctypes.c_int, [_H, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp, _sz, ctypes.c_int, _u32, _dp, _vp,
                               ctypes.POINTER(Stats)]),
    "sv_vqe_step": (ctypes.c_int, [_H, _u64, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp, _sz, ctypes.c_int, _dp, _vp,
                                   _vp, ctypes.POINTER(Stats)]),
    "sv_plan_qsu": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _sz, ctypes.c_int, ctypes.POINTER(Options),
                                   _vp, ctypes.POINTER(_vp)]),
    "sv_plan_evc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _sz, ctypes.c_int, ctypes.POINTER(Options),
                                   _vp, ctypes.POINTER(_vp)]),
    "sv_plan_info": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "sv_plan_order": (ctypes.c_int, [_vp, _i32p]),
    "sv_plan_tile": (ctypes.c_int, [_vp, _i32, _i32p, _i32p, _u64p, _i32p, _i32p, _i32p]),
    "sv_plan_pass": (ctypes.c_int, [_vp, _i32, _i32p, _u64p, _i32p, _i32p]),
    "sv_plan_tile_intra": (ctypes.c_int, [_vp, _i32, _u64p]),
    "sv_plan_free": (None, [_vp]),
    "sv_batch_run": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                    _u64, ctypes.POINTER(Options), _vp, _vp, _vp, _vp, ctypes.POINTER(Stats)]),
    "sv_expect_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _sz, _dp, _vp, _vp]),
    "sv_autotune": (ctypes.c_int, [_H, _u64, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp, _sz, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(Options), _dp]),
    "sv_batch_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                         _u64, ctypes.POINTER(Options), _vp, ctypes.c_int, ctypes.POINTER(Options),
                                         _dp]),
    "sv_synchronize": (ctypes.c_int, [_H]),
    "sv_last_error": (ctypes.c_char_p, []),
    "sv_version": (ctypes.c_char_p, []),
}

for _name, (_res, _args) in EXPORTS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def merge_stats(a: "Stats", b: "Stats") -> "Stats":
    """Stats of two consecutive calls (a QSU call, then an EVC call) as one:
    per-kind launches, bytes and times add; plan counters come from the call
    that owns them."""
    m = Stats()
    ctypes.memmove(ctypes.byref(m), ctypes.byref(a), ctypes.sizeof(Stats))
    for f in ("evc_tiles", "evc_qrs", "evc_passes", "hpsi_passes", "adj_passes"):
        setattr(m, f, getattr(a, f) + getattr(b, f))
    m.launches = a.launches + b.launches
    m.plan_cache_hit = int(a.plan_cache_hit and b.plan_cache_hit)
    m.plan_ms = a.plan_ms + b.plan_ms
    for i in range(len(m.kernels)):
        m.kernels[i] = a.kernels[i] + b.kernels[i]
        m.bytes[i] = a.bytes[i] + b.bytes[i]
        m.ms[i] = a.ms[i] + b.ms[i]
    return m


def _check(status):
    if status != SV_OK:
        raise SvError(status, _lib.sv_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_options(dtype=C64) -> Options:
    o = Options()
    _lib.sv_options_default(dtype, ctypes.byref(o))
    return o


def gate_array(circ) -> np.ndarray:
    """sv_gate records (7 int32 each) from a workloads.Circuit."""
    g = np.zeros((circ.m, 7), np.int32)
    g[:, 0] = circ.kinds
    g[:, 1:5] = circ.qubits
    g[:, 5] = circ.param
    g[:, 6] = circ.mat
    return np.ascontiguousarray(g)


def pauli_array(x, z) -> np.ndarray:
    p = np.zeros((len(x), 2), np.uint64)
    p[:, 0] = np.asarray(x, np.uint64)
    p[:, 1] = np.asarray(z, np.uint64)
    return np.ascontiguousarray(p)


def hamiltonian_arrays(ham):
    """(sv_pauli records, float64 coefficients) from a workloads.Hamiltonian."""
    from .workloads import pauli_masks
    x, z = pauli_masks(ham)
    return pauli_array(x, z), np.ascontiguousarray(ham.coeffs, np.float64)


def _mats(circ):
    if circ.mats is None or circ.mats.size == 0:
        return None, 0
    m = np.ascontiguousarray(circ.mats, np.float64)
    return m, m.size // 2


class StateVector:
    """One simulator handle: n qubits, 2^g virtual chunks, complex64 or
    complex128 state in a torch tensor on the current CUDA device."""

    def __init__(self, n: int, g: int, dtype: int = C64, device=None, options: Options | None = None):
        import torch
        self.torch = torch
        self.n, self.g, self.dtype = n, g, dtype
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        h = _H()
        with torch.cuda.device(self.device):
            _check(_lib.sv_create(n, g, dtype, ctypes.byref(h)))
        self._h = h
        tdt = torch.complex64 if dtype == C64 else torch.complex128
        self.state = torch.zeros(1 << n, dtype=tdt, device=self.device)
        self.lam = None
        _check(_lib.sv_attach_state(self._h, ctypes.c_void_p(self.state.data_ptr()),
                                    self.state.numel() * self.state.element_size()))
        self.set_stream(torch.cuda.current_stream(self.device))
        if options is not None:
            self.set_options(options)
        self.last_stats = Stats()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.sv_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    # ---------------------------------------------------------------- setup
    def set_stream(self, stream):
        _check(_lib.sv_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def set_options(self, opt: Options):
        _check(_lib.sv_set_options(self._h, ctypes.byref(opt)))

    def options(self) -> Options:
        o = Options()
        _check(_lib.sv_get_options(self._h, ctypes.byref(o)))
        return o

    def ensure_lambda(self):
        if self.lam is None:
            self.lam = self.torch.empty_like(self.state)
            _check(_lib.sv_attach_lambda(self._h, ctypes.c_void_p(self.lam.data_ptr()),
                                         self.lam.numel() * self.lam.element_size()))

    # ---------------------------------------------------------------- state
    def reset(self, index: int = 0):
        _check(_lib.sv_reset_basis(self._h, int(index)))

    def set_state(self, vec):
        """vec: complex array (numpy host or torch) in logical order."""
        t = self.torch
        if isinstance(vec, np.ndarray):
            arr = np.ascontiguousarray(vec, np.complex64 if self.dtype == C64 else np.complex128)
            _check(_lib.sv_set_state(self._h, _ptr(arr), 0))
        else:
            v = vec.to(device=self.device, dtype=self.state.dtype).contiguous()
            _check(_lib.sv_set_state(self._h, ctypes.c_void_p(v.data_ptr()), 1))
            t.cuda.current_stream(self.device).synchronize()

    def get_state(self, logical: bool = True) -> np.ndarray:
        out = np.empty(1 << self.n, np.complex64 if self.dtype == C64 else np.complex128)
        _check(_lib.sv_get_state(self._h, _ptr(out), 0, 1 if logical else 0))
        return out

    def permutation(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        _check(_lib.sv_get_permutation(self._h, out.ctypes.data_as(_i32p)))
        return out

    # ---------------------------------------------------------------- work
    def apply_circuit(self, circ, params, schedule: int = LAZY) -> Stats:
        gates = gate_array(circ)
        params = np.ascontiguousarray(params, np.float64)
        mats, nm = _mats(circ)
        st = Stats()
        _check(_lib.sv_apply_circuit(self._h, _ptr(gates), circ.m, _ptr(params), params.size,
                                     _ptr(mats) if mats is not None else None, nm, schedule, ctypes.byref(st)))
        self.last_stats = st
        return st

    def expect(self, ham=None, schedule: int = LAZY, keep_layout: bool = False, paulis=None, coeffs=None,
               per_term: bool = True):
        if ham is not None:
            paulis, coeffs = hamiltonian_arrays(ham)
        coeffs = np.ascontiguousarray(coeffs, np.float64)
        e = ctypes.c_double(0.0)
        pt = np.zeros(len(coeffs), np.float64) if per_term else None
        st = Stats()
        _check(_lib.sv_expect(self._h, _ptr(paulis), _ptr(coeffs), len(coeffs), schedule,
                              KEEP_LAYOUT if keep_layout else 0, ctypes.byref(e),
                              _ptr(pt) if pt is not None else None, ctypes.byref(st)))
        self.last_stats = st
        return e.value, pt

    def apply_hamiltonian(self, ham=None, paulis=None, coeffs=None):
        """Returns (energy, lambda = H psi as a torch tensor in the physical layout)."""
        if ham is not None:
            paulis, coeffs = hamiltonian_arrays(ham)
        coeffs = np.ascontiguousarray(coeffs, np.float64)
        self.ensure_lambda()
        out = self.torch.empty_like(self.state)
        e = ctypes.c_double(0.0)
        st = Stats()
        _check(_lib.sv_apply_hamiltonian(self._h, _ptr(paulis), _ptr(coeffs), len(coeffs),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.byref(e), ctypes.byref(st)))
        self.last_stats = st
        return e.value, out

    def grad(self, circ, params, ham=None, schedule: int = LAZY, forward_done: bool = False, paulis=None,
             coeffs=None):
        if ham is not None:
            paulis, coeffs = hamiltonian_arrays(ham)
        coeffs = np.ascontiguousarray(coeffs, np.float64)
        gates = gate_array(circ)
        params = np.ascontiguousarray(params, np.float64)
        mats, nm = _mats(circ)
        self.ensure_lambda()
        e = ctypes.c_double(0.0)
        g = np.zeros(params.size, np.float64)
        st = Stats()
        _check(_lib.sv_grad(self._h, _ptr(gates), circ.m, _ptr(params), params.size,
                            _ptr(mats) if mats is not None else None, nm, _ptr(paulis), _ptr(coeffs), len(coeffs),
                            schedule, FORWARD_DONE if forward_done else 0, ctypes.byref(e), _ptr(g),
                            ctypes.byref(st)))
        self.last_stats = st
        return e.value, g

    def vqe_step(self, init_index: int, circ, params, ham=None, schedule: int = LAZY, paulis=None, coeffs=None,
                 per_term: bool = False):
        if ham is not None:
            paulis, coeffs = hamiltonian_arrays(ham)
        coeffs = np.ascontiguousarray(coeffs, np.float64)
        gates = gate_array(circ)
        params = np.ascontiguousarray(params, np.float64)
        mats, nm = _mats(circ)
        self.ensure_lambda()
        e = ctypes.c_double(0.0)
        g = np.zeros(params.size, np.float64)
        pt = np.zeros(len(coeffs), np.float64) if per_term else None
        st = Stats()
        _check(_lib.sv_vqe_step(self._h, int(init_index), _ptr(gates), circ.m, _ptr(params), params.size,
                                _ptr(mats) if mats is not None else None, nm, _ptr(paulis), _ptr(coeffs),
                                len(coeffs), schedule, ctypes.byref(e), _ptr(pt) if pt is not None else None,
                                _ptr(g), ctypes.byref(st)))
        self.last_stats = st
        return e.value, g, pt

    def synchronize(self):
        _check(_lib.sv_synchronize(self._h))

    def autotune(self, circ, params, ham=None, schedule: int = LAZY, init_index: int = 0, reps: int = 1,
                 paulis=None, coeffs=None):
        """sv_autotune: times the step (vqe_step with a Hamiltonian, else the
        circuit alone) per candidate option set, leaves the fastest set on the
        handle and returns (Options, ms)."""
        if ham is not None:
            paulis, coeffs = hamiltonian_arrays(ham)
        nterms = 0
        if coeffs is not None:
            coeffs = np.ascontiguousarray(coeffs, np.float64)
            nterms = len(coeffs)
            self.ensure_lambda()
        gates = gate_array(circ)
        params = np.ascontiguousarray(params, np.float64)
        mats, nm = _mats(circ)
        best = Options()
        ms = ctypes.c_double(0.0)
        _check(_lib.sv_autotune(self._h, int(init_index), _ptr(gates), circ.m, _ptr(params), params.size,
                                _ptr(mats) if mats is not None else None, nm,
                                _ptr(paulis) if nterms else None, _ptr(coeffs) if nterms else None, nterms,
                                schedule, int(reps), ctypes.byref(best), ctypes.byref(ms)))
        return best, ms.value


# -------------------------------------------------------------- host plans --

def _plan_dict(p, n, is_qsu):
    nt, no, npass = _i32(), _i32(), _i32()
    _check(_lib.sv_plan_info(p, ctypes.byref(nt), ctypes.byref(no), ctypes.byref(npass)))
    order = np.zeros(max(no.value, 1), np.int32)
    _check(_lib.sv_plan_order(p, order.ctypes.data_as(_i32p)))
    tiles = []
    for t in range(nt.value):
        b, e, npairs = _i32(), _i32(), _i32()
        lm = _u64()
        pairs = np.zeros(128, np.int32)
        l2p = np.zeros(n, np.int32)
        _check(_lib.sv_plan_tile(p, t, ctypes.byref(b), ctypes.byref(e), ctypes.byref(lm), ctypes.byref(npairs),
                                 pairs.ctypes.data_as(_i32p), l2p.ctypes.data_as(_i32p)))
        im = _u64()
        _check(_lib.sv_plan_tile_intra(p, t, ctypes.byref(im)))
        tiles.append(dict(begin=b.value, end=e.value, local_mask=lm.value,
                          pairs=[(int(pairs[2 * i]), int(pairs[2 * i + 1])) for i in range(npairs.value)],
                          l2p=[int(v) for v in l2p], intra_mask=im.value))
    passes = []
    if is_qsu:
        for i in range(npass.value):
            tile, nops = _i32(), _i32()
            bits = _u64()
            _check(_lib.sv_plan_pass(p, i, ctypes.byref(tile), ctypes.byref(bits), ctypes.byref(nops), None))
            ops = np.zeros(max(nops.value, 1), np.int32)
            _check(_lib.sv_plan_pass(p, i, ctypes.byref(tile), ctypes.byref(bits), ctypes.byref(nops),
                                     ops.ctypes.data_as(_i32p)))
            passes.append(dict(tile=tile.value, bits=bits.value, ops=[int(v) for v in ops[:nops.value]]))
    return dict(order=[int(v) for v in order[:no.value]], tiles=tiles, passes=passes, npasses=npass.value)


def plan_qsu(n: int, g: int, circ, schedule: int = LAZY, options: Options | None = None, l2p=None) -> dict:
    gates = gate_array(circ)
    p = _vp()
    l2 = None if l2p is None else np.ascontiguousarray(l2p, np.int32)
    _check(_lib.sv_plan_qsu(n, g, _ptr(gates), circ.m, schedule,
                            ctypes.byref(options) if options is not None else None,
                            _ptr(l2) if l2 is not None else None, ctypes.byref(p)))
    try:
        return _plan_dict(p, n, True)
    finally:
        _lib.sv_plan_free(p)


def plan_evc(n: int, g: int, x, z, schedule: int = LAZY, options: Options | None = None, l2p=None) -> dict:
    paulis = pauli_array(x, z)
    p = _vp()
    l2 = None if l2p is None else np.ascontiguousarray(l2p, np.int32)
    _check(_lib.sv_plan_evc(n, g, _ptr(paulis), len(paulis), schedule,
                            ctypes.byref(options) if options is not None else None,
                            _ptr(l2) if l2 is not None else None, ctypes.byref(p)))
    try:
        return _plan_dict(p, n, False)
    finally:
        _lib.sv_plan_free(p)


def expect_noalloc(state, n: int, dtype: int, paulis, coeffs, stream=None, per_term: bool = True):
    """sv_expect_noalloc on a device tensor `state` (index order): returns
    (energy, per-term values).  Allocates no device memory."""
    import torch
    want = torch.complex64 if dtype == C64 else torch.complex128
    if not state.is_cuda or state.dtype != want or not state.is_contiguous() or state.numel() != (1 << n):
        raise ValueError(f"expect_noalloc: state must be a contiguous CUDA {want} tensor of 2^{n} amplitudes")
    coeffs = np.ascontiguousarray(coeffs, np.float64)
    paulis = np.ascontiguousarray(paulis, np.uint64)
    e = ctypes.c_double(0.0)
    pt = np.zeros(len(coeffs), np.float64) if per_term else None
    with torch.cuda.device(state.device):     # the C side works on the current device
        st = torch.cuda.current_stream(state.device) if stream is None else stream
        _check(_lib.sv_expect_noalloc(ctypes.c_void_p(state.data_ptr()), n, dtype, _ptr(paulis), _ptr(coeffs),
                                      len(coeffs), ctypes.byref(e), _ptr(pt) if pt is not None else None,
                                      ctypes.c_void_p(st.cuda_stream)))
    return e.value, pt


def _batch_arrays(circuits, params_list, ham, paulis, coeffs):
    if ham is not None:
        paulis, coeffs = hamiltonian_arrays(ham)
    coeffs = np.ascontiguousarray(coeffs, np.float64)
    gates = np.ascontiguousarray(np.concatenate([gate_array(c) for c in circuits]), np.int32)
    gate_off = np.zeros(len(circuits) + 1, np.int32)
    gate_off[1:] = np.cumsum([c.m for c in circuits])
    params = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64) for p in params_list]), np.float64)
    param_off = np.zeros(len(circuits) + 1, np.int32)
    param_off[1:] = np.cumsum([len(p) for p in params_list])
    return gates, gate_off, params, param_off, paulis, coeffs


def batch_run(n: int, dtype: int, circuits, params_list, ham=None, paulis=None, coeffs=None, init_index: int = 0,
              options: Options | None = None, stream=None):
    """sv_batch_run over independent states: circuits[b] (workloads.Circuit)
    with params_list[b].  Returns (energies, list of gradients, times_ns
    (batch, 2) start/end, Stats)."""
    import torch
    gates, gate_off, params, param_off, paulis, coeffs = _batch_arrays(circuits, params_list, ham, paulis, coeffs)
    batch = len(circuits)
    energies = np.zeros(batch, np.float64)
    grads = np.zeros(max(params.size, 1), np.float64)
    times = np.zeros(2 * batch, np.float64)
    st = Stats()
    s = torch.cuda.current_stream() if stream is None else stream
    _check(_lib.sv_batch_run(n, dtype, batch, _ptr(gates), _ptr(gate_off), _ptr(params), _ptr(param_off),
                             _ptr(paulis), _ptr(coeffs), len(coeffs), int(init_index),
                             ctypes.byref(options) if options is not None else None, ctypes.c_void_p(s.cuda_stream),
                             _ptr(energies), _ptr(grads), _ptr(times), ctypes.byref(st)))
    gl = [grads[param_off[b]:param_off[b + 1]].copy() for b in range(batch)]
    return energies, gl, times.reshape(batch, 2), st


def batch_autotune(n: int, dtype: int, circuits, params_list, ham=None, paulis=None, coeffs=None,
                   init_index: int = 0, options: Options | None = None, stream=None, reps: int = 2):
    """sv_batch_autotune: returns (fastest Options, device ms of one batched
    launch with them)."""
    import torch
    gates, gate_off, params, param_off, paulis, coeffs = _batch_arrays(circuits, params_list, ham, paulis, coeffs)
    s = torch.cuda.current_stream() if stream is None else stream
    best = Options()
    ms = ctypes.c_double(0.0)
    _check(_lib.sv_batch_autotune(n, dtype, len(circuits), _ptr(gates), _ptr(gate_off), _ptr(params),
                                  _ptr(param_off), _ptr(paulis), _ptr(coeffs), len(coeffs), int(init_index),
                                  ctypes.byref(options) if options is not None else None,
                                  ctypes.c_void_p(s.cuda_stream), int(reps), ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


def version() -> str:
    return _lib.sv_version().decode()
