#!/usr/bin/env python3
"""Benchmark of one VQE iteration -- QSU, EVC and the adjoint gradient --
under the lazy qubit-reordering schedule on one GB300 (arXiv 2410.04252).

Default workload: n = 32 qubits, 2^6 virtual chunks, complex64 (32 GiB per
state), hardware-efficient ansatz of 6 layers (570 gates, 384 parameters),
1024 random Pauli strings; eager (ad hoc QR) schedule measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on stdout (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica on its own GPU (the path has no exchange step on one
GPU); the timed region is bracketed by barriers and the max over ranks is
taken.  --impl reference times the CPU oracle on a bounded sample of the
same workload on the host cores, scaled to one full iteration.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VQE iter time (QSU+EVC+adjoint grad), HBM GB/s vs peak; lazy-QR vs eager"
BATCH_METRIC = "batched VQE iterations (QSU+EVC+adjoint grad), per-state latency and throughput"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--n", type=int, default=0, help="override qubit count (smaller runs)")
    ap.add_argument("--eager-steps", type=int, default=1)
    ap.add_argument("--eager-warmup", type=int, default=1)
    ap.add_argument("--no-eager", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--plan-table", action="store_true", help="print plan-level QR counts (host only) and exit")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: default options")
    ap.add_argument("--cpu-n", type=int, default=22, help="qubits of the measured same-size oracle baseline")
    ap.add_argument("--ref-n", type=int, default=20, help="qubits of the reference arm's per-step oracle sample")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline workload (no further configs in the line)")
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--low-bits", type=int, default=0)
    ap.add_argument("--evc-low-bits", type=int, default=0)
    ap.add_argument("--evc-span", type=int, default=-1)
    return ap.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.h", "api.cu", "plan.cpp", "sv_internal.h"):
        with open(os.path.join(ROOT, "paper_2410_04252_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kind: str):
    """Per-launch DRAM bytes of `kind` in `workload` from the committed ncu
    summary, or None if absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get("workloads", {}).get(workload, {}).get(kind)
    if not k:
        return None
    return k.get("dram_bytes_per_full_launch")


# ----------------------------------------------------------------- oracle --

def oracle_sample(cfg_id: int, n_full: int, n_s: int, nterm_sample: int = 16):
    """Time the oracle on a bounded sample and scale it to one full step of
    the workload computed the oracle's way: QSU (gate by gate), EVC (string by
    string) and, for the gradient workload, the parameter-shift gradient
    (1 + 2 * np evaluations of QSU + EVC); each evaluation scaled by
    2^(n_full - n_s), by the gate count and by nterms / nterm_sample."""
    import numpy as np
    import oracle
    from paper_2410_04252_gb300 import workloads as W
    cfg = W.CONFIGS[cfg_id]
    batch = cfg.get("batch", 1)
    # batched workload: one state of the mean depth stands for each state
    layers = (cfg["layers"] + cfg["min_layers"]) // 2 if batch > 1 else cfg["layers"]
    circ = W.make_circuit(cfg, n_s, layers)
    params = W.make_params(cfg_id, circ)
    ham = W.make_hamiltonian(cfg_id, n_s)
    init = W.make_init(cfg, n_s)
    t0 = time.perf_counter()
    psi = oracle.apply_circuit(oracle.basis_state(n_s, init), circ, params)
    t1 = time.perf_counter()
    if ham is not None:
        sub = W.Hamiltonian(n_s, ham.letters[:nterm_sample], ham.coeffs[:nterm_sample])
        oracle.energy(psi, sub)
    t2 = time.perf_counter()
    full_circ = W.make_circuit(cfg, n_full, layers)
    scale = 2.0 ** (n_full - n_s)
    t_qsu = (t1 - t0) * scale * full_circ.m / max(circ.m, 1)
    t_evc = (t2 - t1) * scale * cfg["nterms"] / nterm_sample * (n_full / n_s) if ham is not None else 0.0
    evals = 1 + 2 * full_circ.nparams if cfg["work"] in ("qsu+evc+grad", "batch") else 1
    est_ms = (t_qsu + t_evc) * evals * batch * 1e3
    what = {"qsu": "", "qsu+evc": "", "qsu+evc+grad": " and %d evaluations (energy + parameter-shift gradient)" % evals,
            "batch": " and %d evaluations (energy + parameter-shift gradient) per state, %d states of %d layers"
                     % (evals, batch, layers)}
    sample = (f"oracle FP64 QSU of the same ansatz at n={n_s} ({circ.m} gates)"
              + (f" + EVC of {nterm_sample} of the {cfg['nterms']} strings" if ham is not None else "")
              + f", {t2 - t0:.2f} s; scaled by 2^{n_full - n_s}, gate count"
              + (", string count" if ham is not None else "") + what[cfg["work"]])
    return est_ms, sample, t2 - t0


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def oracle_step(cfg_id, n_s):
    """One real step of the oracle's own path at n_s qubits (QSU gate by
    gate, then EVC of every string; for the batched workload one state of the
    mean depth): wall ms and a description."""
    import oracle
    from paper_2410_04252_gb300 import workloads as W
    cfg = W.CONFIGS[cfg_id]
    layers = (cfg["layers"] + cfg["min_layers"]) // 2 if cfg.get("batch", 1) > 1 else cfg["layers"]
    circ = W.make_circuit(cfg, n_s, layers)
    params = W.make_params(cfg_id, circ)
    ham = W.make_hamiltonian(cfg_id, n_s)
    t0 = time.perf_counter()
    psi = oracle.apply_circuit(oracle.basis_state(n_s, W.make_init(cfg, n_s)), circ, params)
    if ham is not None:
        oracle.energy(psi, ham)
    ms = (time.perf_counter() - t0) * 1e3
    what = ("oracle FP64 QSU (%d gates) + EVC of all %d strings of the workload at n=%d (no gradient)"
            % (circ.m, len(ham.coeffs) if ham is not None else 0, n_s))
    return ms, what


def workload_config(cfg_id, n, world):
    """The workload's identity as both arms print it in `config` (host data
    only: no library call)."""
    from paper_2410_04252_gb300 import workloads as W
    cfg = W.CONFIGS[cfg_id]
    circ = W.make_circuit(cfg, n)
    state_gb = (1 << n) * (8 if cfg["dtype"] == "c64" else 16) / 1e9
    return {"workload": cfg["name"], "n": n, "g": cfg["g"], "layers": cfg["layers"], "gates": circ.m,
            "params": circ.nparams, "nterms": cfg["nterms"], "schedule": "lazy", "state_GB": state_gb,
            "l2": "inputs larger than L2 (state %.1f GB)" % state_gb,
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, timed for real on the
    host cores, each step one run of the workload's QSU + EVC at --ref-n
    qubits (a bounded sample of the workload: same ansatz, depth and
    Hamiltonian, fewer qubits).  Its full-size estimate (scaled to n and with
    the parameter-shift gradient) is reported beside, labelled as one."""
    rank, local, world = rank_info()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from paper_2410_04252_gb300 import workloads as W
    cfg = W.CONFIGS[args.config]
    n_full = args.n or cfg["n"]
    n_s = min(args.ref_n, n_full)
    for _ in range(args.warmup):
        oracle_step(args.config, min(n_s, 14))
    vals = []
    what = ""
    for _ in range(args.steps):
        ms, what = oracle_step(args.config, n_s)
        vals.append(ms)
    ms = statistics.median(vals)
    est_ms, est_how, _ = oracle_sample(args.config, n_full, n_s)
    metric, value, unit, hib = METRIC, ms, "ms", False
    if cfg["work"] == "batch":
        metric = BATCH_METRIC
        value, unit, hib = 1.0 / (ms * 1e-3), "states/s", True
    config = workload_config(args.config, n_full, world) if cfg["work"] != "batch" else {"workload": cfg["name"]}
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": hib,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "sample": {"n": n_s, "what": what},
            "cpu_baseline": {"value": value, "unit": unit, "cores": omp_threads(), "kind": "oracle",
                             "sample": what + " (measured, median of the timed steps)"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "estimate_full_workload_ms": est_ms, "estimate_how": est_how}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours --

def reduce_times(dev_ms, wall_ms, steps, world, dist=None, device="cpu"):
    """Max over ranks of the device and wall times of the timed region.
    Every rank runs its own replica of the iteration, so one iteration takes
    the same time at any rank count: returns (device ms, wall ms, device ms
    per iteration of one replica, whole-job iterations per second = steps x
    ranks over the device time, wall ms per iteration of one replica)."""
    import torch
    t = torch.tensor([dev_ms, wall_ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, wall_ms = float(t[0]), float(t[1])
    return dev_ms, wall_ms, dev_ms / steps, steps * world / (dev_ms * 1e-3), wall_ms / steps


def _timed_region(fn, stream, clocks):
    """Run fn() between CUDA events on `stream` (synchronised on both sides),
    with nvidia-smi clocks sampled meanwhile.  Returns (device ms, wall ms,
    clocks, fn's result)."""
    import torch
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    ev0.record(stream)
    res = fn()
    ev1.record(stream)
    ev1.synchronize()
    wall = (time.perf_counter() - w0) * 1e3
    clk = clocks.stop() if clocks is not None else None
    return ev0.elapsed_time(ev1), wall, clk, res


class Workload:
    """One workload (configuration, qubit count, dtype) on one handle: its
    seeded inputs in pinned host memory and the step of its path through the
    public API (reset, QSU, EVC and, for the gradient workload, lambda and
    the reverse sweep)."""

    def __init__(self, cfg_id, n=None, dtype=None, opt_args=None, work=None):
        import numpy as np
        import torch
        from paper_2410_04252_gb300 import sv
        from paper_2410_04252_gb300 import workloads as W
        self.sv, self.np = sv, np
        self.cfg_id = cfg_id
        self.cfg = cfg = W.CONFIGS[cfg_id]
        self.n = n or cfg["n"]
        self.g = cfg["g"]
        self.dtype = dtype if dtype is not None else (sv.C64 if cfg["dtype"] == "c64" else sv.C128)
        self.work = work or cfg["work"]
        self.circ = W.make_circuit(cfg, self.n)
        ham = W.make_hamiltonian(cfg_id, self.n)
        paulis, coeffs = sv.hamiltonian_arrays(ham) if ham is not None else (None, np.zeros(0))
        # the step's host inputs live in pinned memory (copied to the device
        # by every call through the public API)
        self.params = torch.from_numpy(W.make_params(cfg_id, self.circ)).pin_memory().numpy()
        self.coeffs = torch.from_numpy(np.ascontiguousarray(coeffs, np.float64)).pin_memory().numpy()
        self.paulis = None
        if paulis is not None:
            self.paulis = torch.from_numpy(np.ascontiguousarray(paulis).view(np.int64)).pin_memory().numpy().view(
                np.uint64)
        self.init = W.make_init(cfg, self.n)
        opt = sv.default_options(self.dtype)
        a = opt_args
        if a is not None:
            if a.tile_bits:
                opt.tile_bits = a.tile_bits
            if a.low_bits:
                opt.low_bits = a.low_bits
            if a.evc_low_bits:
                opt.evc_low_bits = a.evc_low_bits
            if a.evc_span >= 0:
                opt.evc_span = a.evc_span
        opt.profile = 1
        self.opt = opt
        self.sim = sv.StateVector(self.n, self.g, self.dtype, options=opt)
        if self.work == "qsu+evc+grad":
            self.sim.ensure_lambda()

    def step(self, schedule):
        """One step; stats of all its calls merged into sim.last_stats.
        Returns (energy, gradient)."""
        sim, sv = self.sim, self.sv
        if self.work == "qsu+evc+grad":
            e, gr, _ = sim.vqe_step(self.init, self.circ, self.params, paulis=self.paulis, coeffs=self.coeffs,
                                    schedule=schedule)
            return e, gr
        sim.reset(self.init)
        st = sim.apply_circuit(self.circ, self.params, schedule)
        e = 0.0
        if self.work == "qsu+evc":
            e, _ = sim.expect(paulis=self.paulis, coeffs=self.coeffs, schedule=schedule)
            st = sv.merge_stats(st, sim.last_stats)
        else:
            sim.synchronize()
        sim.last_stats = st
        return e, self.np.zeros(0)

    def bytes_io(self):
        """Host->device and device->host bytes of one step through the API."""
        h2d = 2 * self.params.nbytes + (self.coeffs.nbytes + self.paulis.nbytes if self.paulis is not None else 0)
        d2h = 16 + (8 * self.params.size if self.work == "qsu+evc+grad" else 0)
        return h2d, d2h

    def close(self):
        import torch
        self.sim.close()
        del self.sim
        torch.cuda.empty_cache()


def measure(wl, schedule, steps, warmup, clocks=None):
    """Warm-up, then `steps` timed steps of one schedule: device and wall time
    per step, per-kernel-kind launches / time / algorithmic bytes, counts."""
    import torch
    sv = wl.sv
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for _ in range(warmup):
        wl.step(schedule)
    warm_s = time.perf_counter() - t0
    agg = {k: [0, 0.0, 0.0] for k in sv.KERNEL_KINDS}
    out = {}

    def body():
        launches = 0
        e = gr = None
        for _ in range(steps):
            e, gr = wl.step(schedule)
            st = wl.sim.last_stats
            launches += st.launches
            for i, k in enumerate(sv.KERNEL_KINDS):
                agg[k][0] += st.kernels[i]
                agg[k][1] += st.bytes[i]
                agg[k][2] += st.ms[i]
            out["counts"] = dict(qsu_tiles=st.qsu_tiles, qsu_qrs=st.qsu_qrs, qsu_passes=st.qsu_passes,
                                 evc_tiles=st.evc_tiles, evc_qrs=st.evc_qrs, evc_passes=st.evc_passes,
                                 hpsi_passes=st.hpsi_passes, adj_passes=st.adj_passes)
        return launches, e, gr

    dev_ms, wall_ms, clk, (launches, e, gr) = _timed_region(body, stream, clocks)
    out.update(dev_ms=dev_ms, wall_ms=wall_ms, clocks=clk, launches=launches, energy=e, grad=gr, agg=agg,
               warm_s=warm_s, steps=steps, warmup=warmup)
    return out


def kernel_table(agg, steps, peak, peak_src, workload=""):
    """Per-kind summary and the dominant kind's roofline entry."""
    kinds = {}
    total = max(sum(v[2] for v in agg.values()), 1e-9)
    for k, (cnt, byts, ms) in agg.items():
        if cnt:
            kinds[k] = {"launches_per_step": cnt / steps, "ms_per_step": ms / steps, "share": ms / total,
                        "algorithmic_GBps": (byts / (ms * 1e-3) / 1e9) if ms > 0 and byts > 0 else None,
                        "bytes_per_launch": byts / cnt,
                        "frac_of_measured_hbm": ((byts / (ms * 1e-3) / 1e9) / peak) if ms > 0 and byts > 0 else None}
    dom = max((k for k in kinds if agg[k][1] > 0), key=lambda k: agg[k][2])
    cnt, byts, ms = agg[dom]
    achieved = byts / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src, "traffic": ncu_traffic(workload, dom)}
    return kinds, roof


def other_schedule(wl, schedule, steps, warmup, ref):
    """The same step under another schedule: time per step, QR counts and the
    energy (and gradient) difference from the lazy step."""
    import numpy as np
    m = measure(wl, schedule, steps, warmup)
    c = m["counts"]
    d = {"ms_per_step": m["dev_ms"] / steps, "qsu_qrs": c["qsu_qrs"], "evc_qrs": c["evc_qrs"],
         "qsu_passes": c["qsu_passes"], "evc_passes": c["evc_passes"], "steps": steps, "warmup": warmup,
         "energy_diff_vs_lazy": abs(m["energy"] - ref["energy"])}
    if m["grad"] is not None and m["grad"].size:
        d["grad_maxdiff_vs_lazy"] = float(np.max(np.abs(m["grad"] - ref["grad"])))
    return d


def extra_workload(cfg_id, steps, warmup, peak, peak_src, local, dtype=None, eager=True):
    """A further workload of the benchmark on this GPU:
    its own timed region, clocks, roofline of its dominant kernel, end-to-end
    time and, for QSU / EVC workloads, the eager schedule beside it."""
    from paper_2410_04252_gb300 import sv
    wl = Workload(cfg_id, dtype=dtype)
    try:
        m = measure(wl, sv.LAZY, steps, warmup, ClockSampler(local))
        kinds, roof = kernel_table(m["agg"], steps, peak, peak_src,
                                   wl.cfg["name"] if dtype is None else wl.cfg["name"].replace("c64", "c128"))
        h2d, d2h = wl.bytes_io()
        state_gb = (1 << wl.n) * (8 if wl.dtype == sv.C64 else 16) / 1e9
        d = {"workload": wl.cfg["name"] if dtype is None else wl.cfg["name"].replace("c64", "c128"),
             "metric": METRIC, "value": m["dev_ms"] / steps, "unit": "ms", "ms_per_step": m["dev_ms"] / steps,
             "higher_is_better": False, "steps": steps, "warmup": warmup,
             "dtype": "c64 (f32 math, f64 accumulation)" if wl.dtype == sv.C64 else "c128 (f64)",
             "config": {"n": wl.n, "g": wl.g, "gates": wl.circ.m, "params": wl.circ.nparams,
                        "nterms": len(wl.coeffs), "work": wl.work, "schedule": "lazy", "state_GB": state_gb,
                        "l2": "inputs larger than L2 (state %.1f GB)" % state_gb},
             "roofline": roof, "kernels": kinds, "counts": m["counts"], "clocks": m["clocks"],
             "gpu_launches": m["launches"], "energy": m["energy"],
             "e2e": {"value": m["wall_ms"] / steps, "unit": "ms", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h, "how": "wall clock around the public calls of the step"}}
        if eager:
            d["eager"] = other_schedule(wl, sv.EAGER, 1, 1, m)
            d["eager"]["speedup_lazy_over_eager"] = d["eager"]["ms_per_step"] / d["ms_per_step"]
        return d
    finally:
        wl.close()


def same_n_baseline(cfg_id, n_s, args):
    """The oracle timed for real on the host cores at a size it finishes in
    seconds (QSU gate by gate + the full Hamiltonian string by string, FP64),
    beside the library at the same size: its whole step and its QSU + EVC
    alone (the oracle's work), both device-timed."""
    import oracle
    from paper_2410_04252_gb300 import sv
    from paper_2410_04252_gb300 import workloads as W
    oracle.build()
    cfg = W.CONFIGS[cfg_id]
    circ = W.make_circuit(cfg, n_s)
    params = W.make_params(cfg_id, circ)
    ham = W.make_hamiltonian(cfg_id, n_s)
    t0 = time.perf_counter()
    psi = oracle.apply_circuit(oracle.basis_state(n_s, W.make_init(cfg, n_s)), circ, params)
    t1 = time.perf_counter()
    e_orc = oracle.energy(psi, ham) if ham is not None else 0.0
    t2 = time.perf_counter()
    out = {"n": n_s, "cores": omp_threads(), "oracle_qsu_ms": (t1 - t0) * 1e3, "oracle_evc_ms": (t2 - t1) * 1e3,
           "measured_ms": (t2 - t0) * 1e3, "oracle_energy": e_orc,
           "what": "oracle FP64 QSU (%d gates) + EVC of all %d strings at n=%d, no gradient"
                   % (circ.m, len(ham.coeffs) if ham is not None else 0, n_s)}
    for work, key in (("qsu+evc", "gpu_same_n_qsu_evc_ms"), (cfg["work"], "gpu_same_n_step_ms")):
        wl = Workload(cfg_id, n=n_s, work=work)
        try:
            m = measure(wl, sv.LAZY, 5, 3)
            out[key] = m["dev_ms"] / 5
            if work == "qsu+evc":
                out["gpu_energy_diff_vs_oracle"] = abs(m["energy"] - e_orc)
        finally:
            wl.close()
    out["speedup_same_n_qsu_evc"] = out["measured_ms"] / out["gpu_same_n_qsu_evc_ms"]
    return out


def run_ours(args):
    import numpy as np
    import torch
    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2410_04252_gb300 import sv

    peak, peak_src = measured_peaks()
    wl = Workload(args.config, n=args.n or None, opt_args=args)
    n, g, dtype, opt = wl.n, wl.g, wl.dtype, wl.opt
    t_setup = time.perf_counter()
    for _ in range(args.warmup):
        wl.step(sv.LAZY)
    plan_s = time.perf_counter() - t_setup
    if dist is not None:
        dist.barrier()
    m = measure(wl, sv.LAZY, args.steps, 0, ClockSampler(local))
    if dist is not None:
        dist.barrier()
    dev_ms, wall_ms, ms_per_step, job_iters_per_s, e2e_value = reduce_times(m["dev_ms"], m["wall_ms"], args.steps,
                                                                             world, dist, "cuda")
    value = ms_per_step
    eager = direct = hier = ldiag = None
    if not args.no_eager:
        eager = other_schedule(wl, sv.EAGER, args.eager_steps, args.eager_warmup, m)
        eager["speedup_lazy_over_eager"] = eager["ms_per_step"] / ms_per_step
    if not args.no_direct:
        # no virtual-chunk constraint (not the paper's method): the single-GPU optimum
        direct = other_schedule(wl, sv.DIRECT, 1, 1, m)
        direct["lazy_over_direct"] = ms_per_step / direct["ms_per_step"]
        if g >= 3:
            # hierarchical tiling (Alg. 4/5, 8 chunks per node) on the same GPU
            ho = wl.sim.options()
            ho.intra_bits = 3
            wl.sim.set_options(ho)
            hier = other_schedule(wl, sv.HIER, 1, 1, m)
            hier["intra_bits"] = 3
            ho.intra_bits = 0
            wl.sim.set_options(ho)
        # diagonal gates exempt from locality (not the paper's method)
        ldiag = other_schedule(wl, sv.LAZY_DIAG, 1, 1, m)
    e, gr = m["energy"], m["grad"]
    h2d, d2h = wl.bytes_io()
    cfg, circ, coeffs = wl.cfg, wl.circ, wl.coeffs
    wl.close()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    kinds, roof = kernel_table(m["agg"], args.steps, peak, peak_src, cfg["name"] if n == cfg["n"] else "")
    cpu = None
    if not args.no_cpu:
        n_s = min(args.cpu_n, n)
        same = same_n_baseline(args.config, n_s, args)
        est_ms, sample, _ = oracle_sample(args.config, n, min(n_s, 22))
        cpu = {"value": same["measured_ms"], "unit": "ms", "cores": same["cores"], "kind": "oracle",
               "sample": same["what"] + " (measured); the same size on this GPU: gpu_same_n_qsu_evc_ms for the "
                                        "same work, gpu_same_n_step_ms for the whole step",
               "measured_ms": same["measured_ms"], "n": n_s, "same_n": same,
               "estimate_full_step_ms": est_ms, "estimate_how": sample}

    extras = {}
    if args.config == 3 and not args.n and not args.headline_only and world == 1:
        for cid in (1, 2):
            extras["cfg%d" % cid] = extra_workload(cid, 3, 2, peak, peak_src, local)
        extras["cfg4"] = run_batch(args, emit=False)
        extras["cfg3_c128"] = extra_workload(3, 2, 1, peak, peak_src, local, dtype=sv.C128, eager=False)

    state_gb = (1 << n) * (8 if dtype == sv.C64 else 16) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (f32 math, f64 accumulation)" if dtype == sv.C64 else "c128 (f64)",
        "data": "synthetic",
        "config": workload_config(args.config, n, world),
        "options": {"tile_bits": opt.tile_bits, "low_bits": opt.low_bits, "evc_low_bits": opt.evc_low_bits,
                    "evc_span": opt.evc_span},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "how": {"qsu+evc+grad": "wall clock around the public vqe_step call (host params/Hamiltonian in, "
                               "energy+grad out)",
                        "qsu+evc": "wall clock around reset + apply_circuit + expect (host params/Hamiltonian "
                                   "in, energy out)",
                        "qsu": "wall clock around reset + apply_circuit + synchronize (host params in)"}[cfg["work"]]},
        "gpu_launches": m["launches"],
        "replicas": {"n": world, "iterations_per_s": job_iters_per_s,
                     "how": "every rank runs its own replica; value is one replica's time per iteration"},
        "clocks": m["clocks"],
        "kernels": kinds,
        "counts": m["counts"],
        "eager": eager,
        "direct": direct,
        "hier": hier,
        "lazy_diag": ldiag,
        "energy": e,
        "plan_and_warmup_s": plan_s,
        "configs": extras or None,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args, emit=True):
    """Batched workload: 256 independent n=18 states, HEA of 2..8 layers with
    per-state parameters, one shared 512-string random Hamiltonian; QSU,
    lambda/energy and adjoint gradient of every state in one persistent
    graph-captured launch."""
    import numpy as np
    import torch
    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    from paper_2410_04252_gb300 import sv
    from paper_2410_04252_gb300 import workloads as W
    cfg = W.CONFIGS[4]
    n = args.n or cfg["n"]
    states = W.batch_states(cfg["batch"], n, cfg["layers"], cfg["min_layers"])
    circs = [W.hea_circuit(n, layers) for layers, _ in states]
    params = [p for _, p in states]
    ham = W.make_hamiltonian(4, n)
    paulis, coeffs = sv.hamiltonian_arrays(ham)
    opt = sv.default_options(sv.C64)
    tuned_ms = None
    if not args.no_autotune:
        # tile size k, CTA size and fusion depth picked by the autotuner
        opt, tuned_ms = sv.batch_autotune(n, sv.C64, circs, params, paulis=paulis, coeffs=coeffs, reps=2)
    for _ in range(args.warmup):
        sv.batch_run(n, sv.C64, circs, params, paulis=paulis, coeffs=coeffs, options=opt)
    clocks = ClockSampler(local)
    clocks.start()
    dev_ms, lat = [], []
    w0 = time.perf_counter()
    for _ in range(args.steps):
        e, g, t, st = sv.batch_run(n, sv.C64, circs, params, paulis=paulis, coeffs=coeffs, options=opt)
        dev_ms.append(st.ms[sv.K_BATCH])
        lat.extend(((t[:, 1] - t[:, 0]) * 1e-6).tolist())
    wall_ms = (time.perf_counter() - w0) * 1e3 / args.steps
    clk = clocks.stop()
    ms = statistics.median(dev_ms)
    lat.sort()
    # algorithmic HBM bytes of one batched launch: per state 2S per gate pass
    # (QSU), 2S + 3S per later H|psi> pass, 4S per adjoint pass (S = 2^n * 8)
    S = float(1 << n) * 8
    npass = {}
    for c in circs:
        if c.m not in npass:
            npass[c.m] = sv.plan_qsu(n, 0, c, sv.LAZY, opt)["npasses"]
    hp = st.hpsi_passes
    byts = sum(6 * S * npass[c.m] for c in circs) + len(circs) * S * (2 + 3 * max(hp - 1, 0))
    peak, peak_src = measured_peaks()
    achieved = byts / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu:
        # one evaluation timed for real at the workload's own n (a state of the
        # mean depth: QSU gate by gate + EVC of every string); the oracle's
        # iteration is 2 np + 1 such evaluations (parameter-shift gradient)
        ms1, what = oracle_step(4, n)
        layers = (cfg["layers"] + cfg["min_layers"]) // 2
        npar = W.make_circuit(cfg, n, layers).nparams
        evals = 2 * npar + 1
        cpu = {"value": 1.0 / (ms1 * 1e-3 * evals), "unit": "states/s", "cores": omp_threads(), "kind": "oracle",
               "measured_ms_one_evaluation": ms1,
               "sample": "%s: %.1f ms measured; one VQE iteration of the oracle = %d evaluations "
                         "(energy + parameter-shift gradient of %d parameters)" % (what, ms1, evals, npar)}
    line = {
        "metric": BATCH_METRIC,
        "value": cfg["batch"] / (ms * 1e-3), "unit": "states/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (f32 math, f64 accumulation)", "data": "synthetic",
        "config": {"workload": cfg["name"], "n": n, "states": cfg["batch"], "layers": "2..8",
                   "nterms": len(coeffs), "launches_per_step": st.launches, "graph_captured": True,
                   "l2": "inputs larger than L2: psi and lambda per resident CTA, %d SMs x 2 x %.0f MiB" % (
                       torch.cuda.get_device_properties(local).multi_processor_count, S / 2**20),
                   "tile_bits": opt.tile_bits, "threads": opt.threads, "fuse_max": opt.fuse_max,
                   "autotuned": tuned_ms is not None},
        "roofline": {"bound": "hbm", "kernel": "batch", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "traffic": ncu_traffic(cfg["name"], "batch") if n == cfg["n"] else None},
        "cpu_baseline": cpu,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "max": lat[-1]},
        "e2e": {"value": cfg["batch"] / (wall_ms * 1e-3), "unit": "states/s",
                "h2d_bytes_per_step": int(sum(p.nbytes for p in params) + paulis.nbytes + coeffs.nbytes),
                "d2h_bytes_per_step": int(8 * (cfg["batch"] + sum(len(p) for p in params))),
                "how": "wall clock around sv_batch_run (plans, buffers, graph launch, copies)"},
        "gpu_launches": st.launches * args.steps,
        "clocks": clk,
    }
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def plan_table(args):
    """Plan-level QR counts of the QSU experiment (Sec. V-B-1): GateFabric
    circuits (4-qubit blocks as one operation, and split into the double
    excitation and two Givens rotations), n = 20..36, 4n layers, 32 chunks
    (g = 5), flat vs hierarchical (8 chunks per node: 3 intra qubits) vs the
    ad hoc rule; host planning only, with its time."""
    from paper_2410_04252_gb300 import sv
    from paper_2410_04252_gb300 import workloads as W
    g, nintra = 5, 3
    rows = []
    for n in range(20, 37, 2):
        for form, make in (("blocks", W.fabric_blocks_circuit), ("split", W.fabric_circuit)):
            c = make(n, 4 * n)
            hopt = sv.default_options()
            hopt.intra_bits = nintra
            row = {"n": n, "form": form, "ops": c.m}
            for name, sched, opt in (("flat", sv.LAZY, None), ("hier", sv.HIER, hopt), ("adhoc", sv.EAGER, None)):
                t0 = time.perf_counter()
                p = sv.plan_qsu(n, g, c, sched, opt)
                row[name + "_plan_s"] = time.perf_counter() - t0
                row[name + "_qrs"] = sum(1 for t in p["tiles"] if t["pairs"])
                if name == "hier":
                    inter = [(t["local_mask"] | t["intra_mask"]) for t in p["tiles"]]
                    row["hier_inter_qrs"] = sum(1 for i in range(1, len(inter))
                                                if inter[i] != inter[i - 1] and p["tiles"][i]["pairs"])
            row["adhoc_over_flat"] = row["adhoc_qrs"] / max(row["flat_qrs"], 1)
            rows.append(row)
    # diagonal exemption (RZ / CZ never ask for a QR) vs the paper's lazy plan,
    # random RY / RZ / CZ circuits of 20n gates
    drows = []
    for n in range(20, 37, 4):
        c = W.random_circuit(n, 20 * n, 4000 + n, (W.RY, W.RZ, W.CZ))
        row = {"n": n, "ops": c.m}
        for name, sched in (("lazy", sv.LAZY), ("lazy_diag", sv.LAZY_DIAG), ("adhoc", sv.EAGER)):
            p = sv.plan_qsu(n, g, c, sched)
            row[name + "_qrs"] = sum(1 for t in p["tiles"] if t["pairs"])
        drows.append(row)
    # EVC (Sec. V-B-2): Alg. 6 with diagonalization vs the index-order ad hoc
    # rule, JW-shaped Hamiltonians of 4096 strings on 32 chunks
    erows = []
    for n in range(20, 37, 4):
        h = W.jw_hamiltonian(n, 4096, 2000 + n)
        x, z = W.pauli_masks(h)
        row = {"n": n, "strings": len(h.coeffs)}
        for name, sched in (("lazy", sv.LAZY), ("adhoc", sv.EAGER)):
            t0 = time.perf_counter()
            p = sv.plan_evc(n, g, x, z, sched)
            row[name + "_plan_s"] = time.perf_counter() - t0
            row[name + "_qrs"] = sum(1 for t in p["tiles"] if t["pairs"])
        row["adhoc_over_lazy"] = row["adhoc_qrs"] / max(row["lazy_qrs"], 1)
        erows.append(row)
    print(json.dumps({"table": "QSU QR counts, flat vs hierarchical vs ad hoc (plan level)", "g": g,
                      "n_intra": nintra, "layers": "4n", "rows": rows,
                      "evc_table": "EVC QR counts, Alg. 6 lazy vs index-order ad hoc, JW-shaped 4096 strings",
                      "evc_rows": erows,
                      "diag_table": "QSU QR counts with diagonal gates exempt, random RY/RZ/CZ circuits",
                      "diag_rows": drows}), flush=True)
    return 0


def main():
    args = parse()
    if args.plan_table:
        return plan_table(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 4:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
