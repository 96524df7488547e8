#!/usr/bin/env python
"""Benchmark of the low-rank stabilizer-decomposition hot path on GB300.

One step = one pass of the whole path over one batch of the QAOA workload: n = 50
qubits, QAOA p = 1 on a seeded degree-4 Max-E3LIN2 instance (gamma = 0.3, beta = 0.2;
264 CX, 150 H and 116 rotation slots), sparsified to chi = 2^20 terms:
  init_terms -> apply_clifford -> amplitude (B = 4096 uniform x) -> norm_estimate
  (L = 512) -> sample chain starts -> chains_init (C = 256) -> Metropolis (T = 64
  steps of the workload's 10^4 per chain).
Units per step: chi-term amplitude evaluations = chi * (B + C * (T + 1)).
`value` is device-resident throughput (inputs already in HBM); `e2e` runs the same
step through the public API with host buffers and the host<->device copies inside
the timed region.  L2 is flushed (256 MB write) before every timed step.  The same
step on the n = 40 random Clifford+T workload (chi = 2^16) is a side study.  Prints
one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "χ-term amplitude evals/s"
UNIT = "term-amplitude evals/s"

# step shapes: batch B, equatorial states L, chains C, Metropolis steps T per step
SHAPES = {
    "qaoa": dict(B=4096, L=512, C=256, T=64),
    "mid": dict(B=4096, L=256, C=256, T=16),
    "qaoa_small": dict(B=2048, L=64, C=64, T=2, chi=1 << 16),   # profiling case
    "qaoa_pi4": dict(B=4096, L=512, C=256, T=64),   # the paper's beta = pi/4 line (Clifford mixer)
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrstab", choices=["lrstab", "reference"])
    ap.add_argument("--workload", default="qaoa", choices=["qaoa", "mid"],
                    help="headline workload (default: the n=50 QAOA step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sampler-study", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the side studies (n=40 step, batching, gadgets, prefixes, marginals, GEMMs)")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: chi = 2^16 terms of the QAOA decomposition, B = 2048, L = 64, "
                         "C = 64, T = 2 (for ncu captures; not a bench line)")
    ap.add_argument("--mlp-gemm-only", action="store_true",
                    help="run only the MADE network tensor-core study (n=64, H=2048, 16384 rows) and "
                         "print its JSON (for ncu captures of the GEMM kernels; not a bench line)")
    ap.add_argument("--hs-marginals", action="store_true",
                    help="only the single-qubit marginals of the 40-qubit hidden shift (2/4/6 CCZ)")
    ap.add_argument("--hidden-shift-chains", action="store_true",
                    help="only the hidden shift's chain study (time for term-sampled chains to reach s)")
    ap.add_argument("--config5-graph", action="store_true",
                    help="only config 5's eight-circuit step, uncaptured and as one CUDA graph")
    ap.add_argument("--hs-sum8-chains", action="store_true",
                    help="only the chains on the 2^24-term hidden shift (1024 chains, 206 GB of Pauli states)")
    ap.add_argument("--qaoa-apply-only", action="store_true",
                    help="run only apply_clifford on the n=50 QAOA circuit at chi = 2^16, twice, and "
                         "print its times (for ncu captures; not a bench line)")
    ap.add_argument("--metropolis-only", action="store_true",
                    help="run only chain starts and 2 x 16 Metropolis steps at chi = 2^16 (n = 40, or "
                         "n = 50 with --workload qaoa), and print their times (for ncu captures; not a "
                         "bench line)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------
# algorithmic work per unit (integer 32-bit op equivalents; 64-bit word op = 2)
# ---------------------------------------------------------------------------------
GATE_OPS = {"S": 4, "SDG": 4, "Z": 2, "CZ": 4, "CX": 12}


def clifford_ops_per_term(n, low, formula=False):
    """Expected integer ops per term of the lowered circuit.

    formula=False (the kernel's count): an H on a qubit no earlier gate has touched
    acts on |0> and needs no row pass (no fan-out, a = 0), so it is counted at its
    constant part (40); every other H or projector at 30n + 40.  formula=True: every
    H and projector at 30 n + 40, the per-gate figure of the hot-path table."""
    import numpy as np
    from paper_1808_00128_gb300 import lrstab
    inv = {v: k for k, v in lrstab.OP.items()}
    h_ops = 30 * n + 40
    touched = set()

    def gate_cost(g):
        name = inv[int(g["op"])]
        q = int(g["q"])
        if name in ("H", "P0", "P1"):
            cost = h_ops if (formula or q in touched or name != "H") else 40
            touched.add(q)
            return cost
        touched.add(q)
        if name in ("CX", "CZ"):
            touched.add(int(g["r"]))
        return GATE_OPS.get(name, 0)

    total = 0.0
    for g in low.gates:
        if inv[int(g["op"])] == "SLOT":
            s = low.slots[int(g["r"])]
            nc = int(s["n_choices"])
            w = np.hypot(s["c_re"][:nc], s["c_im"][:nc])
            w = w / w.sum()
            snap = set(touched)
            acc = 0.0
            for j in range(nc):
                touched.clear()
                touched.update(snap)
                sub = low.kgates[s["k_off"][j]: s["k_off"][j] + s["k_len"][j]]
                acc += w[j] * sum(gate_cost(k) for k in sub)
            touched.clear()
            touched.update(snap)
            for j in range(nc):
                for k in low.kgates[s["k_off"][j]: s["k_off"][j] + s["k_len"][j]]:
                    touched.add(int(k["q"]))
            total += acc
        else:
            total += gate_cost(g)
    return total


def amplitude_ops_per_unit(n, mean_popcount_x, formula=False):
    """Integer ops per (x, term).  Kernel count: Four-Russians lookups, 4 word ops per
    4-row chunk, 8 ceil(n/4) + 16.  Formula of the hot-path table: 10 |x| + 30 (one
    row step per set bit of x)."""
    if formula:
        return 10.0 * mean_popcount_x + 30.0
    return 8.0 * ((n + 3) // 4) + 16.0


def norm_ops_per_unit(n, vw, max_folds):
    """32-bit integer ops per (A, term) of the norm estimate, by the path a term takes.
    K path (n - |v| > max_folds): the two products of K = G^T (A+J) G, 8 n^2, plus the
    pairwise elimination on |v| variables, 4 |v|^2.  Change-of-variables path: the rows
    of A + J and the lifted rows, 8 n, one rank-2 update per folded constraint, 5 n
    each, and the same elimination, 4 |v|^2.  max_folds = -1 gives the hot-path
    table's formula 8 n^2 + 4 |v|^2 for every term."""
    import numpy as np
    vw = np.asarray(vw)
    m = n - vw
    return np.where(m <= max_folds, 8 * n + 5 * m * n + 4 * vw ** 2, 8 * n * n + 4 * vw ** 2)


def metropolis_bytes(chi, C, T, n, accept=0.5, lookahead=1):
    """Algorithmic HBM bytes of T steps of C chains: the 16-byte state of every (chain,
    term) read, written back for accepted moves, and the rows F_j, M_j of every term
    (16 n bytes per term per step).  With two steps per pass the state is read once per
    pass and written back when either of its two moves was accepted."""
    one = chi * C * (16 + 16 * accept) + chi * 16 * n
    if lookahead == 1:
        return T * one
    two = chi * C * (16 + 16 * (1 - (1 - accept) ** 2)) + 2 * chi * 16 * n
    return (T // 2) * two + (T % 2) * one


def units_per_step(chi, B, C, T):
    return chi * (B + C * (T + 1))


def launches_per_step(T, lookahead=1):
    """Library kernels one step launches: init, apply, amplitude + reduce, norm (prep,
    equatorial draws, norm, reduce), chain starts, chains_init (amplitude with Pauli
    states, reduce, chain scalars), Metropolis (set, first, graphs of 16 steps with
    2 launches per pass of `lookahead` steps and an advance node, the remaining steps,
    out)."""
    g, r = divmod(T, 16)
    per_graph = 2 * (16 // lookahead) + 1
    rest = 2 * (r // lookahead + r % lookahead)
    return 1 + 1 + 2 + 4 + 1 + 3 + (2 + g * per_graph + rest + 1)


# DRAM bytes per launch of the dominant kernel (ncu: dram__bytes_read.sum +
# dram__bytes_write.sum), per unit of work, with the hash of the kernel source the
# capture ran; `traffic` is reported only while that source is unchanged.
TRAFFIC = {
    # k_norm<13, 7> on the profiling case (n = 50 QAOA, chi = 2^16, L = 64): 34,172,672 B
    # read + 185,088 B written per launch for 2^16 x 64 (A, term) units
    "norm_estimate": {"bytes_per_unit": (34172672 + 185088) / (65536 * 64),
                      "source": "paper_1808_00128_gb300/csrc/k_norm.cu", "sha16": "8f42b33d2b5067dc",
                      "profile": "profiles/k_norm_n50_chi65536_L64.md"},
}


def source_sha16(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(phase, units):
    t = TRAFFIC.get(phase)
    if not t:
        return None, None
    if source_sha16(t["source"]) != t["sha16"]:
        return None, f"{t['profile']} (kernel changed since the capture)"
    return t["bytes_per_unit"] * units, t["profile"]


# ---------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------
# CPU oracle timing: a bounded sample of the step, spread over the host cores
# ---------------------------------------------------------------------------------
def _oracle_worker(args):
    """One host process: build `k` terms of the decomposition (from term alpha0),
    evaluate their amplitudes at n_x strings and their equatorial inner products with
    n_a states; returns the seconds of each phase and its unit counts."""
    cfg_name, alpha0, k, n_x, n_a = args
    from oracle import decomp
    from oracle import estimators as E
    from paper_1808_00128_gb300 import workloads
    cfg = workload_config(cfg_name)
    n, ops = cfg["n"], cfg["ops"]
    xs = [int(x) for x in workloads.random_bitstrings(n, n_x, seed=workloads.SEED_BASE + 50 + alpha0)]
    t0 = time.perf_counter()
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=cfg["chi"], mode=cfg["mode"], seed=cfg["seed"],
                                                 alphas=range(alpha0, alpha0 + k))
    t1 = time.perf_counter()
    for t, b in zip(terms, coefs):
        for x in xs:
            b * t.amplitude(x)
    t2 = time.perf_counter()
    for l in range(n_a):
        A = E.draw_A(n, 7 + alpha0, l)
        for t in terms:
            E.inner_equatorial(t, A)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2, k, k * n_x, k * n_a


def workload_config(name):
    from paper_1808_00128_gb300 import workloads
    if name == "qaoa":
        return workloads.config_qaoa()
    if name == "qaoa_pi4":
        cfg = workloads.config_qaoa(beta=math.pi / 4)
        cfg["name"] = "qaoa_e3lin2_n50_beta_pi4"
        return cfg
    return workloads.config_mid()


class OracleTimer:
    """The oracle as it stands, run on all host cores by a spawn-started process
    pool (safe after CUDA initialisation).  A sample gives per-unit single-core times
    of term building, amplitude evaluation and equatorial inner products; the step's
    oracle time is the step's units times those, divided by the parallelism the pool
    achieved (busy seconds / wall seconds)."""

    def __init__(self, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers or max(1, os.cpu_count() or 1)
        self.pool = cf.ProcessPoolExecutor(max_workers=self.workers, mp_context=mp.get_context("spawn"))
        list(self.pool.map(_noop, range(self.workers)))          # start the workers

    def sample(self, cfg_name, k, n_x, n_a, alpha0=0):
        t0 = time.perf_counter()
        res = list(self.pool.map(_oracle_worker, [(cfg_name, alpha0 + w * k, k, n_x, n_a)
                                                  for w in range(self.workers)]))
        wall = time.perf_counter() - t0
        tb = sum(r[0] for r in res) / sum(r[3] for r in res)
        ta = sum(r[1] for r in res) / sum(r[4] for r in res)
        ti = sum(r[2] for r in res) / sum(r[5] for r in res)
        busy = sum(r[0] + r[1] + r[2] for r in res)
        return {"t_build": tb, "t_amp": ta, "t_inner": ti, "parallel": busy / wall, "wall": wall, "busy": busy}

    def close(self):
        self.pool.shutdown()


def _noop(_):
    import oracle.estimators  # noqa: F401  (import cost paid before timing)
    return 0


class COracleTimer:
    """The C restatement of the oracle (oracle/c/chform_oracle.c) on all host threads:
    wall times of building k terms alone, with their amplitudes at n_x strings, and with
    their equatorial inner products with n_a states give per-unit times of the whole
    machine."""

    def __init__(self, name):
        from oracle import fast
        cfg = workload_config(name)
        self.cfg = cfg
        self.prep = fast.Prepared(cfg["n"], cfg["ops"], cfg["chi"], cfg["mode"], cfg["seed"])
        self.threads = max(1, os.cpu_count() or 1)

    def sample(self, k, n_x, n_a, alpha0=0):
        from oracle import estimators as E
        from paper_1808_00128_gb300 import workloads
        n = self.cfg["n"]
        xs = [int(x) for x in workloads.random_bitstrings(n, n_x, seed=workloads.SEED_BASE + 50 + alpha0)]
        As = [E.draw_A(n, 7 + alpha0, l) for l in range(n_a)]
        t0 = time.perf_counter()
        self.prep.sums([], [], alpha0=alpha0, count=k, threads=self.threads)
        t1 = time.perf_counter()
        self.prep.sums(xs, [], alpha0=alpha0, count=k, threads=self.threads)
        t2 = time.perf_counter()
        self.prep.sums([], As, alpha0=alpha0, count=k, threads=self.threads)
        t3 = time.perf_counter()
        tb = (t1 - t0) / k
        return {"t_build": tb, "t_amp": max(t2 - t1 - (t1 - t0), 0.0) / (k * n_x),
                "t_inner": max(t3 - t2 - (t1 - t0), 0.0) / (k * n_a), "parallel": 1.0, "wall": t3 - t0}


def oracle_step_seconds(chi, shape, rates):
    serial = chi * (rates["t_build"] + (shape["B"] + shape["C"] * (shape["T"] + 1)) * rates["t_amp"]
                    + shape["L"] * rates["t_inner"])
    return serial / max(rates["parallel"], 1.0)


def run_reference(args):
    """The oracle as it stands, timed on the host cores (bounded sample per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    cfg, shape = workload_config(name), SHAPES[name]
    chi = cfg["chi"]
    units = units_per_step(chi, shape["B"], shape["C"], shape["T"])
    timer = COracleTimer(name)
    per = dict(k=4096, n_x=128, n_a=4)
    for w in range(args.warmup):
        timer.sample(alpha0=10000 * w, **per)
    times, vals = [], []
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = timer.sample(alpha0=100000 + 10000 * k, **per)
        times.append(time.perf_counter() - t0)
        vals.append(units / oracle_step_seconds(chi, shape, r))
    value = statistics.median(vals)
    sample = (f"per step: {per['k']} terms of the {cfg['name']} decomposition built by the C restatement "
              f"of the oracle on {timer.threads} host threads, with {per['n_x']} amplitude evaluations and "
              f"{per['n_a']} equatorial inner products per term (exact integer sums); wall times per unit "
              "scaled to one full step (chi terms, chi (B + C (T+1)) amplitude evaluations, chi L inner "
              "products)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "n": cfg["n"], "chi": chi, "batch": shape["B"],
                      "L": shape["L"], "chains": shape["C"], "metropolis_steps": shape["T"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": timer.threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------------
class StepRunner:
    """One workload's step on one GPU: the context, device buffers and the timed
    phases."""

    PHASES = ["init_terms", "apply_clifford", "amplitude", "norm_estimate", "chains_init", "metropolis"]

    def __init__(self, name, local=0, rank=0, small=False):
        import numpy as np
        import torch
        from paper_1808_00128_gb300 import lrstab, workloads
        self.name = name
        self.cfg = workload_config(name)
        self.shape = dict(SHAPES["qaoa_small" if small else name])
        self.n = self.cfg["n"]
        self.chi_total = self.cfg["chi"]
        self.chi = self.shape.pop("chi", self.chi_total)
        self.seed = self.cfg["seed"] + 1000 * rank          # rank r: its own instance
        self.low = lrstab.lower_circuit(self.n, self.cfg["ops"])
        self.dev = torch.device(f"cuda:{local}")
        B, L, C = self.shape["B"], self.shape["L"], self.shape["C"]
        self.x_host = torch.from_numpy(workloads.random_bitstrings(self.n, B, seed=workloads.SEED_BASE + 40)
                                       .view(np.int64)).pin_memory()
        self.x_dev = self.x_host.to(self.dev)
        self.amp = torch.empty((B, 2), dtype=torch.float64, device=self.dev)
        self.eta = torch.empty(L, dtype=torch.float64, device=self.dev)
        self.x0 = torch.empty(C, dtype=torch.int64, device=self.dev)
        self.xo = torch.empty(C, dtype=torch.int64, device=self.dev)
        self.po = torch.empty(C, dtype=torch.float64, device=self.dev)
        self.sim = lrstab.Simulator(self.n, local)
        self.stream = torch.cuda.current_stream()

    def units(self):
        s = self.shape
        return units_per_step(self.chi, s["B"], s["C"], s["T"])

    @property
    def lookahead(self):
        """Metropolis steps per pass over the Pauli states (the context's knob, read
        while the context is open and kept)."""
        if getattr(self, "_look", None) is None:
            self._look = self.sim.get_tuning("mc_lookahead")
        return self._look

    def step(self, ev=None, idx=0):
        st = self.stream

        def mark(i):
            if ev is not None:
                ev[i].record(st)
        s = self.shape
        mark(0)
        self.sim.init_terms(self.low, self.chi, mode="sparsify", seed=self.seed, chi_total=self.chi_total)
        mark(1)
        self.sim.apply_clifford(self.low.gates)
        mark(2)
        self.sim.amplitude(self.x_dev, out=self.amp)
        mark(3)
        self.sim.norm_estimate(s["L"], seed=1000 + idx, eta=self.eta)
        mark(4)
        self.sim.sample_terms(s["C"], seed=2000 + idx, x=self.x0)
        self.sim.chains_init(self.x0)
        mark(5)
        self.sim.metropolis(s["T"], seed=3000 + idx, x_out=self.xo, p_out=self.po)
        mark(6)

    def tune(self, cache_path=None):
        from paper_1808_00128_gb300 import autotune
        s = self.shape
        return {k: v for k, (v, ms) in autotune.tune(self.sim, x=self.x_dev, L=s["L"], chains=s["C"],
                                                       cache_path=cache_path).items()}

    def timed(self, steps, idx0, flush, world=1):
        import torch
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            self.step(evs[k], idx=idx0 + k)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        per_phase = {p: [] for p in self.PHASES}
        step_ms = []
        for e in evs:
            for i, p in enumerate(self.PHASES):
                per_phase[p].append(e[i].elapsed_time(e[i + 1]))
            step_ms.append(e[0].elapsed_time(e[6]))
        return step_ms, {p: statistics.mean(v) for p, v in per_phase.items()}

    def e2e(self, steps, idx0, flush):
        import torch
        s = self.shape
        amp_h = torch.empty((s["B"], 2), dtype=torch.float64).pin_memory()
        eta_h = torch.empty(s["L"], dtype=torch.float64).pin_memory()
        xo_h = torch.empty(s["C"], dtype=torch.int64).pin_memory()
        po_h = torch.empty(s["C"], dtype=torch.float64).pin_memory()
        ms = []
        for k in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            self.x_dev.copy_(self.x_host, non_blocking=True)
            self.step(idx=idx0 + k)
            amp_h.copy_(self.amp, non_blocking=True)
            eta_h.copy_(self.eta, non_blocking=True)
            xo_h.copy_(self.xo, non_blocking=True)
            po_h.copy_(self.po, non_blocking=True)
            e1.record(self.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        h2d = self.x_host.numel() * 8 + len(self.low.gates) * 4
        d2h = amp_h.numel() * 8 + eta_h.numel() * 8 + xo_h.numel() * 8 + po_h.numel() * 8
        return statistics.mean(ms), h2d, d2h

    def rooflines(self, phase_ms, alu_peak, hbm_peak):
        """Per phase: achieved and fraction of the roofline on the kernel's own op count
        and on the hot-path table's formula."""
        import numpy as np
        n, chi, s = self.n, self.chi, self.shape
        ex = self.sim.export_terms(0, min(chi, 4096))
        vw = np.array([bin(int(v)).count("1") for v in ex["v"]])
        xs = self.x_host.numpy().view(np.uint64)
        xpop = float(np.mean([bin(int(x)).count("1") for x in xs]))
        folds = self.sim.get_tuning("norm_max_folds")
        ops = {
            "apply_clifford": (chi * clifford_ops_per_term(n, self.low), chi * clifford_ops_per_term(n, self.low, True)),
            "amplitude": (chi * s["B"] * amplitude_ops_per_unit(n, xpop),
                          chi * s["B"] * amplitude_ops_per_unit(n, xpop, True)),
            "norm_estimate": (chi * s["L"] * float(np.mean(norm_ops_per_unit(n, vw, folds))),
                              chi * s["L"] * float(np.mean(norm_ops_per_unit(n, vw, -1)))),
        }
        units = {"apply_clifford": ("term-gates", chi * len(self.low.gates)),
                 "amplitude": ("(x, term)", chi * s["B"]), "norm_estimate": ("(A, term)", chi * s["L"]),
                 "metropolis": ("chain-term-steps", chi * s["C"] * s["T"])}
        rows = {}
        for p, (k_ops, f_ops) in ops.items():
            t = phase_ms[p] * 1e-3
            rows[p] = {"bound": "alu", "achieved": k_ops / t / 1e12, "peak": alu_peak / 1e12, "unit": "Tops/s",
                       "frac": k_ops / t / alu_peak, "frac_formula": f_ops / t / alu_peak, "ms": phase_ms[p],
                       "rate": units[p][1] / t, "rate_unit": units[p][0] + "/s"}
        t = phase_ms["metropolis"] * 1e-3
        # the kernel's own bytes (two steps per pass read the states once) and the
        # hot-path table's one-step-per-pass bytes
        byts = metropolis_bytes(chi, s["C"], s["T"], n, lookahead=self.lookahead)
        byts1 = metropolis_bytes(chi, s["C"], s["T"], n)
        rows["metropolis"] = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                              "frac": byts / t / 1e9 / hbm_peak, "frac_formula": byts1 / t / 1e9 / hbm_peak,
                              "steps_per_pass": self.lookahead,
                              "ms": phase_ms["metropolis"], "ms_per_metropolis_step": phase_ms["metropolis"] / s["T"],
                              "rate": units["metropolis"][1] / t, "rate_unit": units["metropolis"][0] + "/s"}
        return rows

    def error_statement(self):
        """The kernel's per-result bound on |a_gpu - exact chi-sum| over the step's
        batch, relative to max(|a|, ||psi|| 2^{-n/2}) with ||psi||^2 the step's norm
        estimate."""
        import numpy as np
        import torch
        err = torch.empty(self.shape["B"], dtype=torch.float32, device=self.dev)
        a = self.sim.amplitude(self.x_dev, err=err).cpu().numpy()
        err = err.cpu().numpy().astype(np.float64)
        mag = np.hypot(a[:, 0], a[:, 1])
        norm = float(np.sqrt(max(self.eta.mean().item(), 0.0)))
        rel = err / np.maximum(mag, norm * 2.0 ** (-self.n / 2))
        return {"bound_max_rel": float(rel.max()), "bound_median_rel": float(np.median(rel)),
                "norm_estimate": norm ** 2, "relative_to": "max(|a|, ||psi|| 2^{-n/2})"}

    def close(self):
        _ = self.lookahead          # kept for the launch count after the context is gone
        self.sim.close()


def slice_parity(name, local=0, chi=128, alpha0=31337, n_x=64, timer=None):
    """Measured error of the CUDA amplitudes against the oracle's exact Z[zeta8]
    chi-sums on a `chi`-term slice of the workload's decomposition, at strings drawn
    from the slice's terms and uniform strings; also checks the kernel's stated
    bound.  The oracle's terms are built on the host pool."""
    import numpy as np
    import torch
    from oracle import exact
    from paper_1808_00128_gb300 import lrstab, workloads
    cfg = workload_config(name)
    n, ops = cfg["n"], cfg["ops"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode=cfg["mode"], seed=cfg["seed"], alpha0=alpha0, chi_total=cfg["chi"])
    sim.apply_clifford(low.gates)
    xs_t = sim.sample_terms(n_x, seed=77).cpu().numpy().view(np.uint64)
    xs = np.concatenate([xs_t, workloads.random_bitstrings(n, n_x, seed=78)])
    x = torch.from_numpy(xs.view(np.int64)).to(f"cuda:{local}")
    err = torch.empty(len(xs), dtype=torch.float32, device=x.device)
    a = sim.amplitude(x, err=err).cpu().numpy()
    sim.close()
    got = a[:, 0] + 1j * a[:, 1]
    err = err.cpu().numpy().astype(np.float64)
    k = max(1, chi // timer.workers) if timer else chi
    jobs = [(name, alpha0 + i, min(k, alpha0 + chi - (alpha0 + i)), [int(v) for v in xs]) for i in range(0, chi, k)]
    parts = list(timer.pool.map(_exact_slice_worker, jobs)) if timer else [_exact_slice_worker(j) for j in jobs]
    ex = exact.ExactDecomposition(n, ops, cfg["chi"], cfg["mode"])
    want = np.array([exact.to_complex(ex.finish_parts([p[i] for p in parts])) for i in range(len(xs))])
    d = np.abs(got - want)
    coef = ex.l1 / cfg["chi"]
    scale = np.maximum(np.abs(want), coef * np.sqrt(chi) * 2.0 ** (-n / 2))
    return {"workload": f"{cfg['name']} terms {alpha0}..{alpha0 + chi - 1}", "strings": int(len(xs)),
            "max_abs_err": float(d.max()), "max_rel_err": float((d / scale).max()),
            "relative_to": "max(|a|, |b| sqrt(chi_slice) 2^{-n/2})",
            "bound_holds": bool(np.all(d <= err)), "max_err_over_bound": float(np.max(d / np.maximum(err, 1e-300)))}


def _exact_slice_worker(args):
    name, a0, k, xs = args
    from oracle import decomp, exact
    cfg = workload_config(name)
    terms, _, chs = decomp.build_decomposition(cfg["n"], cfg["ops"], chi=cfg["chi"], mode=cfg["mode"],
                                               seed=cfg["seed"], alphas=range(a0, a0 + k))
    ex = exact.ExactDecomposition(cfg["n"], cfg["ops"], cfg["chi"], cfg["mode"])
    return [ex.amplitude_parts(terms, chs, x) for x in xs]


# ---------------------------------------------------------------------------------
# side studies
# ---------------------------------------------------------------------------------

def tau_int(series):
    """Integrated autocorrelation time of a [T][C] series (chain-averaged
    autocorrelation, Sokal's automatic window with c = 5)."""
    import numpy as np
    x = np.asarray(series, float)
    x = x - x.mean(axis=0, keepdims=True)
    T = x.shape[0]
    var = (x * x).mean()
    if var == 0:
        return 1.0
    f = np.fft.rfft(x, n=2 * T, axis=0)
    ac = np.fft.irfft(f * np.conj(f), axis=0)[:T].mean(axis=1)
    rho = ac / ac[0]
    tau = 1.0
    for w in range(1, T):
        tau += 2.0 * rho[w]
        if w >= 5.0 * tau:
            break
    return max(tau, 1.0)


def _cost_table(inst, n):
    """Per-triple (mask, sign) of the E3LIN2 objective C(z) = 1/2 sum d z_u z_v z_w."""
    return [((1 << u) | (1 << v) | (1 << w), d) for (u, v, w), d in inst]


def _parity64(v):
    """Parity of each uint64 (XOR folding)."""
    import numpy as np
    v = v.copy()
    for sh in (32, 16, 8, 4, 2, 1):
        v ^= v >> np.uint64(sh)
    return (v & np.uint64(1)).astype(np.int64)


def _observables(xs, n, table):
    """Cost 2 C(z) (integer), Hamming weight and bits of uint64 strings."""
    import numpy as np
    xs = np.asarray(xs, dtype=np.uint64).reshape(-1)
    bits = ((xs[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.int8)
    cost2 = np.zeros(xs.size, np.int64)
    for mask, d in table:
        # z_u z_v z_w = (-1)^{x_u + x_v + x_w}
        cost2 += d * (1 - 2 * _parity64(xs & np.uint64(mask)))
    return cost2, bits.sum(axis=1), bits


def _tv_hist(a, b_probs, offset, size):
    import numpy as np
    h = np.bincount(a + offset, minlength=size)[:size] / max(a.size, 1)
    return 0.5 * float(np.abs(h - b_probs).sum())


def _run_traced(fn, C, steps, chunk, dev):
    """Run `steps` steps of a sampler in chunks with traces; returns (trace [steps, C]
    on the host, per-chunk cumulative GPU seconds)."""
    import numpy as np
    import torch
    trace = np.empty((steps, C), np.uint64)
    buf = torch.empty((chunk, C), dtype=torch.int64, device=dev)
    t, times, done = 0.0, [], 0
    while done < steps:
        k = min(chunk, steps - done)
        a, b = _ev()
        a.record()
        fn(k, done, buf[:k])
        b.record()
        b.synchronize()
        t += a.elapsed_time(b) * 1e-3
        trace[done:done + k] = buf[:k].cpu().numpy().view(np.uint64)
        done += k
        times.append((done, t))
    return trace, times


def sampler_study(local=0, n=20, chi=1 << 14, C=1024, hidden=512, train_samples=100_000, epochs=20,
                  plain_steps=1500, learned_steps=150, burn=100, chunk=10, tv_targets=(0.05, 0.02, 0.01),
                  ref_steps=0, seed=0, qaoa_instance=False):
    """Plain single-flip Metropolis (Sec. 4.2) against Metropolis-Hastings with the
    learned MADE proposal, on a QAOA Max-E3LIN2 state (gamma 0.3, beta 0.2), at equal
    accuracy and with every cost charged.

    Reference distribution: for n <= 24 the exact P of the sparsified state over all 2^n
    strings (amplitude kernel); otherwise `ref_steps` further steps of plain chains.
    Accuracy: total-variation distance of the pooled samples' cost histogram C(z) to
    the reference, and the largest error of a single-bit marginal.  For each target the
    GPU seconds each sampler needs to get there; ESS/s from the integrated
    autocorrelation of C(z); the learned sampler is charged, besides its own steps, the
    plain steps that produced its training samples and the training itself.
    n = 50 with qaoa_instance=True takes the 50-variable instance of the QAOA workload."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    dev = torch.device(f"cuda:{local}")
    if qaoa_instance:
        cfg = workload_config("qaoa")
        ops, inst, dseed, chi_total = cfg["ops"], cfg["instance"], cfg["seed"], cfg["chi"]
        n = cfg["n"]
    else:
        ops, inst = workloads.qaoa_e3lin2_circuit(n, 4, 0.3, 0.2, workloads.SEED_BASE + 20 + seed)
        dseed, chi_total = workloads.SEED_BASE + 21 + seed, chi
    table = _cost_table(inst, n)
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode="sparsify", seed=dseed, chi_total=chi_total)
    sim.apply_clifford(low.gates)
    off = 2 * len(table) + 1
    size = 2 * off + 1
    x0 = sim.sample_terms(C, seed=7)

    def plain(k, done, buf, step0):
        sim.metropolis(k, seed=11, step0=step0 + done, trace=buf)

    # burn-in of the plain chains
    sim.chains_init(x0)
    sim.metropolis(burn, seed=11)
    # reference
    if n <= 24:
        allx = torch.arange(1 << n, dtype=torch.int64, device=dev)
        amp = sim.amplitude(allx).cpu().numpy()
        P = amp[:, 0] ** 2 + amp[:, 1] ** 2
        P /= P.sum()
        c_all, _, b_all = _observables(np.arange(1 << n, dtype=np.uint64), n, table)
        ref_cost = np.bincount(c_all + off, weights=P, minlength=size)
        ref_bits = (b_all * P[:, None]).sum(axis=0)
        ref_kind = "exact P of the sparsified state (all 2^n strings)"
        del amp, allx
    else:
        rtrace, _ = _run_traced(lambda k, d, b: plain(k, d, b, 10 ** 6), C, ref_steps, chunk, dev)
        rc, _, rb = _observables(rtrace[::2], n, table)
        ref_cost = np.bincount(rc + off, minlength=size) / rc.size
        ref_bits = rb.mean(axis=0)
        ref_kind = f"{ref_steps} steps of {C} plain chains (every 2nd step, {rc.size} samples)"
        sim.chains_init(x0)
        sim.metropolis(burn, seed=11)

    def accuracy(trace, times):
        """Per target: first (steps, GPU seconds) at which the pooled samples reach it."""
        cost, _, bits = _observables(trace, n, table)
        cost = cost.reshape(trace.shape)
        bits = bits.reshape(trace.shape + (n,))
        out = {}
        for tgt in tv_targets:
            hit = None
            for steps, t in times:
                tv = _tv_hist(cost[:steps].reshape(-1), ref_cost, off, size)
                mb = float(np.abs(bits[:steps].reshape(-1, n).mean(axis=0) - ref_bits).max())
                if tv <= tgt and mb <= tgt:
                    hit = {"steps": steps, "gpu_s": t, "tv_cost": tv, "max_bit_err": mb}
                    break
            out[str(tgt)] = hit
        tv_end = _tv_hist(cost.reshape(-1), ref_cost, off, size)
        mb_end = float(np.abs(bits.reshape(-1, n).mean(axis=0) - ref_bits).max())
        return out, tv_end, mb_end, cost

    # plain chains
    ptrace, ptimes = _run_traced(lambda k, d, b: plain(k, d, b, burn), C, plain_steps, chunk, dev)
    t_plain = ptimes[-1][1]
    p_hits, p_tv, p_mb, p_cost = accuracy(ptrace, ptimes)
    tau_p = tau_int(p_cost)
    ess_plain = C * plain_steps / tau_p / t_plain

    # training data: plain-chain states, one every third of an autocorrelation time
    thin = max(1, int(round(tau_p / 3)))
    need_steps = int(np.ceil(train_samples / C)) * thin
    a, b = _ev()
    a.record()
    dtrace = torch.empty((need_steps, C), dtype=torch.int64, device=dev)
    sim.metropolis(need_steps, seed=17, step0=10 ** 7, trace=dtrace)
    data = dtrace[::thin].reshape(-1)[:train_samples].contiguous()
    b.record()
    b.synchronize()
    t_data = a.elapsed_time(b) * 1e-3
    del dtrace
    net = lrstab.MLP(n, hidden, local)
    rng = np.random.default_rng(5)
    lim1, lim2 = 1 / np.sqrt(n), 1 / np.sqrt(hidden)
    net.set_params(dict(W1=rng.uniform(-lim1, lim1, (hidden, n)), b1=rng.uniform(-lim1, lim1, hidden),
                        W2=rng.uniform(-lim2, lim2, (hidden, hidden)), b2=rng.uniform(-lim2, lim2, hidden),
                        W3=rng.uniform(-lim2, lim2, (n, hidden)), b3=rng.uniform(-lim2, lim2, n)))
    bs = 1024
    net.backward(data[:bs].contiguous())   # first launches (module loading) outside the timed region
    _ = data[torch.randperm(data.numel(), device=dev)]   # and the first shuffle (kernel loading)
    torch.cuda.synchronize()
    train_steps = max(1, epochs * data.numel() // bs)
    gen = torch.Generator(device=dev).manual_seed(3)
    a, b = _ev()
    a.record()
    for ep in range(epochs):
        # one gather per epoch; the batches are then contiguous slices (no launch each)
        shuf = data[torch.randperm(data.numel(), device=dev, generator=gen)]
        for it in range(data.numel() // bs):
            net.train_step(shuf[it * bs:(it + 1) * bs], lr=1e-3)
    b.record()
    b.synchronize()
    t_train = a.elapsed_time(b) * 1e-3
    nll = float(net.backward(data[:8192].contiguous()).item())

    # learned proposal
    sim.chains_init(x0)
    lrstab.metropolis_learned(sim, net, 20, seed=13)   # burn-in
    acc = torch.zeros(C, dtype=torch.int64, device=dev)
    ltrace, ltimes = _run_traced(
        lambda k, d, buf: lrstab.metropolis_learned(sim, net, k, seed=13, step0=20 + d, trace=buf, accepts=acc),
        C, learned_steps, chunk, dev)
    t_learned = ltimes[-1][1]
    l_hits, l_tv, l_mb, l_cost = accuracy(ltrace, ltimes)
    tau_l = tau_int(l_cost)
    ess_learned = C * learned_steps / tau_l / t_learned
    overhead = t_data + t_train
    ess_learned_all = C * learned_steps / tau_l / (t_learned + overhead)
    # effective samples above which the learned sampler, overhead included, is faster
    gain = 1.0 / ess_plain - 1.0 / ess_learned
    breakeven = overhead / gain if gain > 0 else None
    matched = {}
    for tgt in tv_targets:
        ph, lh = p_hits[str(tgt)], l_hits[str(tgt)]
        matched[str(tgt)] = {
            "plain_gpu_s": ph["gpu_s"] if ph else None,
            "learned_gpu_s": lh["gpu_s"] if lh else None,
            "learned_gpu_s_with_overhead": (lh["gpu_s"] + overhead) if lh else None,
            "plain_steps": ph["steps"] if ph else None, "learned_steps": lh["steps"] if lh else None}
    # the paper's QAOA run length (Sec. 2.4.1: 10^4 burn-in and 4 x 10^4 sample steps per
    # chain) on these chains: the plain chains' GPU time, and the learned sampler's time,
    # overheads included, for the same number of effective samples
    n_eff = C * 4 * 10 ** 4 / tau_p
    t_plain_run = 5 * 10 ** 4 * t_plain / plain_steps
    t_learned_run = overhead + (20 + n_eff * tau_l / C) * t_learned / learned_steps
    sim.close()
    net.close()
    return {"workload": f"qaoa_e3lin2_n{n}_chi{chi}", "chains": C, "hidden": hidden,
            "paper_run_length": {"effective_samples": n_eff, "plain_gpu_s": t_plain_run,
                                 "learned_gpu_s_with_overhead": t_learned_run,
                                 "speedup": t_plain_run / t_learned_run},
            "observable": "E3LIN2 cost C(z); single-bit marginals", "reference": ref_kind,
            "plain": {"steps": plain_steps, "gpu_s": t_plain, "tau_int": tau_p, "ess_per_s": ess_plain,
                      "tv_cost_end": p_tv, "max_bit_err_end": p_mb},
            "learned": {"steps": learned_steps, "gpu_s": t_learned, "tau_int": tau_l, "ess_per_s": ess_learned,
                        "ess_per_s_with_overhead": ess_learned_all, "tv_cost_end": l_tv, "max_bit_err_end": l_mb,
                        "acceptance": float(acc.sum().item()) / (C * learned_steps),
                        "train_samples": int(data.numel()), "train_steps": int(train_steps), "epochs": epochs,
                        "data_gpu_s": t_data, "train_gpu_s": t_train, "nll": nll},
            "ess_ratio_learned_over_plain": ess_learned / ess_plain,
            "ess_ratio_with_overhead": ess_learned_all / ess_plain,
            "breakeven_effective_samples": breakeven, "matched_tv": matched}


def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def metropolis_only(local=0, C=256, T=16, workload="mid"):
    """Chain starts and two calls of T Metropolis steps at chi = 2^16 terms of the n=40
    workload (or the n=50 QAOA one), C chains; propose launches 17..32 are the second
    call's."""
    import torch
    from paper_1808_00128_gb300 import lrstab
    cfg = workload_config(workload)
    n, chi = cfg["n"], 1 << 16
    low = lrstab.lower_circuit(n, cfg["ops"])
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode="sparsify", seed=cfg["seed"], chi_total=cfg["chi"])
    sim.apply_clifford(low.gates)
    x0 = sim.sample_terms(C, seed=5)
    sim.chains_init(x0)
    ms = []
    for rep in range(2):
        a, b = _ev()
        a.record()
        sim.metropolis(T, seed=6, step0=rep * T)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    sim.close()
    return {"workload": f"{cfg['name']}_chi{chi}_C{C}", "steps": T, "ms": ms}


def qaoa_apply_only(local=0, chi=1 << 16, lanes=(1, 2, 4)):
    """apply_clifford alone on the n=50 QAOA circuit, chi = 2^16, once per lanes-per-term
    value (one launch each, after one warm-up launch)."""
    from paper_1808_00128_gb300 import lrstab
    cfg = workload_config("qaoa")
    low = lrstab.lower_circuit(cfg["n"], cfg["ops"])
    sim = lrstab.Simulator(cfg["n"], local)
    sim.init_terms(low, chi, mode="sparsify", seed=cfg["seed"], chi_total=cfg["chi"])
    sim.apply_clifford(low.gates)
    ms = {}
    for lv in lanes:
        sim.set_tuning("apply_lanes", lv)
        sim.init_terms(low, chi, mode="sparsify", seed=cfg["seed"], chi_total=cfg["chi"])
        a, b = _ev()
        a.record()
        sim.apply_clifford(low.gates)
        b.record()
        b.synchronize()
        ms[lv] = a.elapsed_time(b)
    sim.close()
    return {"workload": f"qaoa_e3lin2_n50_chi{chi}", "apply_ms_by_lanes": ms}


def batch_study(local=0, k=8, seed=0):
    """8 QAOA n=50 circuits (seeds +i) with chi_i = 2^e_i, e_i uniform in 14..20:
    term-gate throughput of one batched launch vs one launch per circuit."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    rng = np.random.default_rng(workloads.SEED_BASE + 5 + seed)
    exps = [int(e) for e in rng.integers(14, 21, size=k)]
    sims, lows, work = [], [], 0
    for i, e in enumerate(exps):
        ops, _ = workloads.qaoa_e3lin2_circuit(50, 4, 0.3, 0.2, workloads.SEED_BASE + 4 + i)
        low = lrstab.lower_circuit(50, ops)
        s = lrstab.Simulator(50, local)
        s.init_terms(low, 1 << e, mode="sparsify", seed=workloads.SEED_BASE + 14 + i)
        sims.append(s)
        lows.append(low)
        work += (1 << e) * len(low.gates)

    def reinit():
        for i, (s, low) in enumerate(zip(sims, lows)):
            s.init_terms(low, 1 << exps[i], mode="sparsify", seed=workloads.SEED_BASE + 14 + i)

    res = {"chi": [1 << e for e in exps]}
    for mode in ("per_circuit", "batched"):
        ts = []
        for rep in range(2):
            reinit()
            torch.cuda.synchronize()
            a, b = _ev()
            a.record()
            if mode == "batched":
                lrstab.apply_clifford_batch(sims, [l.gates for l in lows])
            else:
                for s, low in zip(sims, lows):
                    s.apply_clifford(low.gates)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        res[mode] = {"ms": min(ts), "term_gates_per_s": work / (min(ts) * 1e-3)}
    res["speedup"] = res["per_circuit"]["ms"] / res["batched"]["ms"]
    # amplitudes (B = 4096 uniform strings per circuit): one launch per circuit against
    # one batched launch and one batched reduction
    xs = [torch.from_numpy(workloads.random_bitstrings(50, 4096, seed=workloads.SEED_BASE + 70 + i).view(np.int64))
          .cuda(local) for i in range(k)]
    outs = [torch.empty((4096, 2), dtype=torch.float64, device=xs[0].device) for _ in range(k)]
    amp = {}
    for mode in ("per_circuit", "batched", "per_circuit", "batched"):
        torch.cuda.synchronize()
        a, b = _ev()
        a.record()
        if mode == "batched":
            lrstab.amplitude_batch(sims, xs, outs)
        else:
            for s, x, o in zip(sims, xs, outs):
                s.amplitude(x, out=o)
        b.record()
        b.synchronize()
        amp[mode] = min(amp.get(mode, 1e30), a.elapsed_time(b))
    res["amplitude"] = {"per_circuit_ms": amp["per_circuit"], "batched_ms": amp["batched"],
                        "speedup": amp["per_circuit"] / amp["batched"]}
    for s in sims:
        s.close()
    return res


def gadget_study(local=0, n=30, n_t=14, B=4096):
    """Fixed-sample gadgets (Sec. 2.3.1) against sum-over-Cliffords on the same
    circuit (n=30, 600 Cliffords + 14 T, both exact with 2^14 terms): the gadget form
    works on n + 14 = 44 qubits.  Times apply_clifford and a B-string amplitude batch
    for each, and checks the amplitudes agree."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    ops = workloads.random_clifford_t(n, 600, n_t, seed=workloads.SEED_BASE + 61)
    dev = torch.device(f"cuda:{local}")
    x = torch.from_numpy(workloads.random_bitstrings(n, B, workloads.SEED_BASE + 63).view(np.int64)).to(dev)
    res, amps = {}, {}
    for method in ("sum", "gadget"):
        low = lrstab.lower_circuit(n, ops, method=method)
        chi = low.exact_chi
        sim = lrstab.Simulator(low.n_total, local)
        ts, ta = [], []
        for rep in range(3):
            sim.init_terms(low, chi, mode="exact")
            a, b = _ev()
            a.record()
            sim.apply_clifford(low.gates)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
            a.record()
            out = sim.amplitude(x)
            b.record()
            b.synchronize()
            ta.append(a.elapsed_time(b))
        amps[method] = out.cpu().numpy()
        res[method] = {"qubits": low.n_total, "chi": chi, "gates": len(low.gates),
                       "apply_ms": min(ts), "amplitude_ms": min(ta)}
        sim.close()
    d = amps["sum"] - amps["gadget"]
    res["max_amplitude_difference"] = float(np.abs(d[:, 0] + 1j * d[:, 1]).max())
    res["gadget_over_sum_time"] = ((res["gadget"]["apply_ms"] + res["gadget"]["amplitude_ms"]) /
                                   (res["sum"]["apply_ms"] + res["sum"]["amplitude_ms"]))
    return res


def prefix_study(local=0, sizes=(16, 20)):
    """Prefix sharing on exact n=40 hidden shifts (16 and 20 CCZ slots, chi = 2^16 and
    2^20): the whole circuit per term (the paper's way) vs lrs_apply_circuit_shared,
    which runs each Clifford segment once per distinct choice prefix.  Same terms bit
    for bit (compared on the first and last 4096 terms)."""
    import numpy as np
    from paper_1808_00128_gb300 import lrstab, workloads
    out = []
    for n_ccz in sizes:
        n = 40
        ops, _ = workloads.hidden_shift_circuit(n, n_ccz, workloads.SEED_BASE + 3)
        chi = 1 << n_ccz
        low = lrstab.lower_circuit(n, ops)
        sim = lrstab.Simulator(n, local)
        res = {"workload": f"hidden_shift_n{n}_ccz{n_ccz}", "chi": chi, "gates": len(low.gates)}
        ex = {}
        for name, fn in (("per_term", sim.apply_clifford), ("shared_prefixes", sim.apply_circuit_shared)):
            ts = []
            for rep in range(3):
                sim.init_terms(low, chi, mode="exact")
                a, b = _ev()
                a.record()
                fn(low.gates)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            res[name] = {"ms": min(ts), "term_gates_per_s": chi * len(low.gates) / (min(ts) * 1e-3)}
            ex[name] = (sim.export_terms(0, 4096), sim.export_terms(chi - 4096, 4096))
        res["speedup"] = res["per_term"]["ms"] / res["shared_prefixes"]["ms"]
        res["identical_terms"] = all(np.array_equal(x[k], y[k]) for x, y in zip(ex["per_term"], ex["shared_prefixes"])
                                     for k in x)
        sim.close()
        out.append(res)
    return out


def config5_graph_study(local=0, k=8, B=4096, L=64, C=256, T=16, seed=0):
    """Config 5's eight n = 50 QAOA circuits (seeds +i, chi_i = 2^e_i with e_i uniform
    in 14..20) through the whole path as one step: terms re-initialised (new
    sparsification), gate updates in one batched launch, B amplitudes per circuit in
    one batched launch, an L-state norm estimate, C chain starts and T Metropolis
    steps per circuit.  The step runs as uncaptured calls and as one CUDA graph
    captured from the same calls; reported: both step times, and whether every output
    of the replay (amplitudes, eta, chain starts, final strings and P(x)) equals the
    uncaptured step's bit for bit."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    dev = torch.device(f"cuda:{local}")
    rng = np.random.default_rng(workloads.SEED_BASE + 5 + seed)
    exps = [int(e) for e in rng.integers(14, 21, size=k)]
    sims, lows = [], []
    for i, e in enumerate(exps):
        ops, _ = workloads.qaoa_e3lin2_circuit(50, 4, 0.3, 0.2, workloads.SEED_BASE + 4 + i)
        low = lrstab.lower_circuit(50, ops)
        s = lrstab.Simulator(50, local)
        s.init_terms(low, 1 << e, mode="sparsify", seed=workloads.SEED_BASE + 14 + i)
        sims.append(s)
        lows.append(low)
    gates = [l.gates for l in lows]
    xs = [torch.from_numpy(workloads.random_bitstrings(50, B, seed=workloads.SEED_BASE + 70 + i).view(np.int64))
          .to(dev) for i in range(k)]
    amps = [torch.empty((B, 2), dtype=torch.float64, device=dev) for _ in sims]
    etas = [torch.empty(L, dtype=torch.float64, device=dev) for _ in sims]
    x0s = [torch.empty(C, dtype=torch.int64, device=dev) for _ in sims]
    xos = [torch.empty(C, dtype=torch.int64, device=dev) for _ in sims]
    pos = [torch.empty(C, dtype=torch.float64, device=dev) for _ in sims]
    outs = amps + etas + x0s + xos + pos

    def step():
        for i, s in enumerate(sims):
            s.reinit_terms(seed=workloads.SEED_BASE + 14 + i)
        lrstab.apply_clifford_batch(sims, gates)
        lrstab.amplitude_batch(sims, xs, amps)
        for i, s in enumerate(sims):
            s.norm_estimate(L, seed=200 + i, eta=etas[i])
            s.sample_terms(C, seed=300 + i, x=x0s[i])
            s.chains_init(x0s[i])
            s.metropolis(T, seed=400 + i, x_out=xos[i], p_out=pos[i])

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = _ev()
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                                   # sizes every buffer, sets kernel attributes
    torch.cuda.current_stream().wait_stream(side)
    eager_ms = timed(step)
    ref = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for o in outs:
        o.zero_()
    graph_ms = timed(g.replay)
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    g.reset()
    for s in sims:
        s.close()
    chis = [1 << e for e in exps]
    return {"chi": chis, "B": B, "L": L, "chains": C, "metropolis_steps": T,
            "step_ms_uncaptured": eager_ms, "step_ms_one_graph": graph_ms, "speedup": eager_ms / graph_ms,
            "replay_equals_uncaptured": same,
            "term_amplitude_evals_per_s_graph": sum(chis) * (B + C * (T + 1)) / (graph_ms * 1e-3)}


def hidden_shift_sum8_study(local=0, chi=1 << 24, L=256, K=3):
    """The 40-qubit hidden shift with its 16 CCZ in the 8-term form (prefactor 1/6,
    xi = 16/9) sparsified to chi = 2^24 terms (17 GB of tableau): term set-up and gate
    updates, <s|psi> and the amplitudes at the neighbours of s, the norm estimate and
    the sparsification certificate."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    n = 40
    ops, s = workloads.hidden_shift_circuit(n, 16, workloads.SEED_BASE + 3)
    low = lrstab.lower_circuit(n, ops, "sum8")
    sim = lrstab.Simulator(n, local)
    a, b = _ev()
    a.record()
    sim.init_terms(low, chi, mode="sparsify", seed=77)
    sim.apply_clifford(low.gates)
    b.record()
    b.synchronize()
    t_build = a.elapsed_time(b)
    xs = [s] + [s ^ (1 << j) for j in range(n)]
    x = torch.tensor(np.asarray(xs, dtype=np.uint64).view(np.int64), device=f"cuda:{local}")
    a.record()
    amp = sim.amplitude(x).cpu().numpy()
    b.record()
    b.synchronize()
    eta = sim.norm_estimate(L, seed=5).cpu().numpy()
    cert = lrstab.sparsification_certificate(sim, L, K, seed=6)
    sim.close()
    mags = np.hypot(amp[:, 0], amp[:, 1])
    return {"workload": f"hidden_shift_n40_ccz16_sum8_chi{chi}", "chi": chi, "gates": len(low.gates),
            "init_and_apply_ms": t_build, "amplitude_ms": a.elapsed_time(b),
            "abs_amp_at_shift": float(mags[0]), "max_abs_amp_at_neighbours": float(mags[1:].max()),
            "mean_eta": float(eta.mean()), "sparsification_certificate": cert}


def hidden_shift_sum8_chain_study(local=0, chi=1 << 24, flip_steps=32, learned_steps=8, chunk=16, hidden=512,
                                  train_samples=100_000, epochs=5, exact_samples=4, L=256, K=3):
    """Chains on the 2^24-term hidden shift (16 CCZ in the 8-term form, prefactor 1/6,
    sparsified; n = 40): 1024 single-flip chains hold 206 GB of Pauli states next to
    the 17 GB tableau.  (a) every chain started at s: how many steps stay at s (P(s)
    is near 1 and every neighbour's amplitude near 0, so a move away is almost never
    accepted); (b) chains started by the term sampler of Sec. 4.2 (a term drawn by
    |b|^2, x from its CH form): chains at s and the first step there, for single flips
    and for Metropolis-Hastings with the learned proposal.  The network is trained on
    `exact_samples` chain-rule samples (end of Sec. 4.3) of the same circuit's exact
    2^16-term decomposition, replicated to 10^5 rows: any proposal leaves the chains'
    target P(x) of the 2^24-term state unchanged, and chain-rule sampling on 2^24 terms
    would take about 256 times as long.  The incremental P(x) of every flip chain is
    compared at the end with |<x|psi>|^2 from the amplitude kernel."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    cfg = workloads.config_hidden_shift()
    n, s, C = cfg["n"], np.uint64(cfg["shift"]), cfg["chains"]
    dev = torch.device(f"cuda:{local}")
    low = lrstab.lower_circuit(n, cfg["ops"], "sum8")
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode="sparsify", seed=77)
    sim.apply_clifford(low.gates)
    x_s = torch.full((C,), int(s), dtype=torch.int64, device=dev)
    x0 = sim.sample_terms(C, seed=31)
    start_at_s = int((x0.cpu().numpy().view(np.uint64) == s).sum())

    def timed(fn):
        a, b = _ev()
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) * 1e-3

    def hits(trace):
        at = trace == s
        found = at.any(axis=0)
        first = np.where(found, at.argmax(axis=0) + 1, -1)
        return int(found.sum()), (int(np.median(first[found])) if found.any() else None)

    def p_check(po, xo):
        amp = sim.amplitude(xo)
        pa = (amp[:, 0] ** 2 + amp[:, 1] ** 2).cpu().numpy()
        pc = po.cpu().numpy()
        return float(np.max(np.abs(pc - pa) / np.maximum(pa, 1e-30)))

    out = {"workload": f"hidden_shift_n40_ccz16_sum8_chi{chi}", "chi": chi, "chains": C,
           "pauli_state_gb": C * chi * 12 / 1e9, "chains_started_at_s": start_at_s}
    xo = torch.empty(C, dtype=torch.int64, device=dev)
    po = torch.empty(C, dtype=torch.float64, device=dev)
    # (a) chains at s
    t_init = timed(lambda: sim.chains_init(x_s))
    trace_s, times_s = _run_traced(lambda k, d, b: sim.metropolis(k, seed=41, step0=d, trace=b), C, flip_steps,
                                   chunk, dev)
    sim.metropolis(0, seed=41, step0=flip_steps, x_out=xo, p_out=po)
    out["from_s"] = {"steps": flip_steps, "chains_init_s": t_init, "gpu_s": times_s[-1][1],
                     "chain_steps_at_s": int((trace_s == s).sum()), "chain_steps": int(trace_s.size),
                     "max_rel_err_p_vs_amplitude": p_check(po, xo)}
    # (b) chains from the term sampler, single flips
    t_init = timed(lambda: sim.chains_init(x0))
    ptrace, ptimes = _run_traced(lambda k, d, b: sim.metropolis(k, seed=42, step0=d, trace=b), C, flip_steps,
                                 chunk, dev)
    sim.metropolis(0, seed=42, step0=flip_steps, x_out=xo, p_out=po)
    p_found, p_med = hits(ptrace)
    out["flip"] = {"steps": flip_steps, "chains_init_s": t_init, "gpu_s": ptimes[-1][1], "chains_at_s": p_found,
                   "median_first_step": p_med, "max_rel_err_p_vs_amplitude": p_check(po, xo)}
    # (b) learned proposal trained on exact samples of the 2^16-term decomposition
    ex = lrstab.Simulator(n, local)
    ex.init_terms(lrstab.lower_circuit(n, cfg["ops"]), cfg["chi"], mode="exact")
    ex.apply_clifford(lrstab.lower_circuit(n, cfg["ops"]).gates)
    work = (lrstab.Simulator(n, local), lrstab.Simulator(n, local))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    samples = []
    for i in range(exact_samples):
        bits, _ = ex.marginal_sample(list(range(n)), L, K, seed=100 + i, work=work)
        samples.append(sum(int(b_) << q for q, b_ in enumerate(bits)))
    torch.cuda.synchronize()
    t_marg = time.perf_counter() - t0
    for w_ in work + (ex,):
        w_.close()
    data = torch.tensor(samples, dtype=torch.int64, device=dev).repeat(train_samples // exact_samples + 1)
    data = data[:train_samples].contiguous()
    net = lrstab.MLP(n, hidden, local)
    rng = np.random.default_rng(5)
    lim1, lim2 = 1 / np.sqrt(n), 1 / np.sqrt(hidden)
    net.set_params(dict(W1=rng.uniform(-lim1, lim1, (hidden, n)), b1=rng.uniform(-lim1, lim1, hidden),
                        W2=rng.uniform(-lim2, lim2, (hidden, hidden)), b2=rng.uniform(-lim2, lim2, hidden),
                        W3=rng.uniform(-lim2, lim2, (n, hidden)), b3=rng.uniform(-lim2, lim2, n)))
    bs = 1024
    net.backward(data[:bs].contiguous())   # first launches and first shuffle outside the timing
    _ = data[torch.randperm(data.numel(), device=dev)]
    torch.cuda.synchronize()
    gen = torch.Generator(device=dev).manual_seed(3)

    def train():
        for ep in range(epochs):
            shuf = data[torch.randperm(data.numel(), device=dev, generator=gen)]
            for it in range(data.numel() // bs):
                net.train_step(shuf[it * bs:(it + 1) * bs], lr=1e-3)
    t_train = timed(train)
    t_init = timed(lambda: sim.chains_init(x0))
    ltrace, ltimes = _run_traced(lambda k, d, b: lrstab.metropolis_learned(sim, net, k, seed=43, step0=d, trace=b),
                                 C, learned_steps, min(chunk, learned_steps), dev)
    net.close()
    sim.close()
    l_found, l_med = hits(ltrace)
    out["learned_on_exact_samples"] = {
        "steps": learned_steps, "chains_init_s": t_init, "gpu_s": ltimes[-1][1], "chains_at_s": l_found,
        "median_first_step": l_med, "chain_steps_at_s": int((ltrace == s).sum()),
        "training": f"{exact_samples} chain-rule samples of the exact 2^16-term decomposition, replicated",
        "train_gpu_s": t_train, "sampler_s": t_marg, "samples_are_the_shift": all(np.uint64(v) == s for v in samples)}
    return out


def hidden_shift_chain_study(local=0, plain_steps=2048, learned_steps=32, chunk=64, hidden=512,
                             train_samples=100_000, epochs=5, exact_samples=4, L=256, K=3):
    """The hidden shift's chains (n = 40, 16 CCZ, exact 2^16-term decomposition of |s>,
    1024 chains): every chain starts at a string sampled from one term (the chain start
    of Sec. 4.2, a term drawn by |b|^2, then x from that CH-form), and each sampler is
    timed until its chains reach the shift s.  P(x) = |<x|psi>|^2 is 1 at s and 0
    elsewhere, so from x != s a single flip sees no gradient (every neighbour has
    P = 0 up to FP32 rounding) and the chain walks blindly on 2^40 strings.  The learned
    proposal is trained (a) on 10^5 states of those flip chains (the protocol of the
    sampler comparison) and (b) on `exact_samples` exact samples of the chain-rule
    marginal sampler (end of Sec. 4.3), replicated to 10^5 rows; its MH steps then
    propose from the network.  Reported: chains at s after each sampler, the first step
    at which they got there, GPU seconds, and for (b) the marginal sampler's seconds."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    cfg = workloads.config_hidden_shift()
    n, chi, s, C = cfg["n"], cfg["chi"], np.uint64(cfg["shift"]), cfg["chains"]
    dev = torch.device(f"cuda:{local}")
    low = lrstab.lower_circuit(n, cfg["ops"])
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    x0 = sim.sample_terms(C, seed=31)
    start_at_s = int((x0.cpu().numpy().view(np.uint64) == s).sum())

    def hits(trace):
        at = trace == s
        found = at.any(axis=0)
        first = np.where(found, at.argmax(axis=0) + 1, -1)
        return int(found.sum()), (int(np.median(first[found])) if found.any() else None)

    # single flips
    sim.chains_init(x0)
    ptrace, ptimes = _run_traced(lambda k, d, b: sim.metropolis(k, seed=41, step0=d, trace=b), C, plain_steps,
                                 chunk, dev)
    p_found, p_med = hits(ptrace)
    plain = {"steps": plain_steps, "gpu_s": ptimes[-1][1], "chains_at_s": p_found, "median_first_step": p_med,
             "distinct_strings_visited": int(np.unique(ptrace).size)}

    def train(data):
        net = lrstab.MLP(n, hidden, local)
        rng = np.random.default_rng(5)
        lim1, lim2 = 1 / np.sqrt(n), 1 / np.sqrt(hidden)
        net.set_params(dict(W1=rng.uniform(-lim1, lim1, (hidden, n)), b1=rng.uniform(-lim1, lim1, hidden),
                            W2=rng.uniform(-lim2, lim2, (hidden, hidden)), b2=rng.uniform(-lim2, lim2, hidden),
                            W3=rng.uniform(-lim2, lim2, (n, hidden)), b3=rng.uniform(-lim2, lim2, n)))
        bs = 1024
        net.backward(data[:bs].contiguous())   # first launches and first shuffle outside the timing
        _ = data[torch.randperm(data.numel(), device=dev)]
        torch.cuda.synchronize()
        gen = torch.Generator(device=dev).manual_seed(3)
        a, b = _ev()
        a.record()
        for ep in range(epochs):
            shuf = data[torch.randperm(data.numel(), device=dev, generator=gen)]
            for it in range(data.numel() // bs):
                net.train_step(shuf[it * bs:(it + 1) * bs], lr=1e-3)
        b.record()
        b.synchronize()
        return net, a.elapsed_time(b) * 1e-3

    def learned(net):
        sim.chains_init(x0)
        ltrace, ltimes = _run_traced(lambda k, d, b: lrstab.metropolis_learned(sim, net, k, seed=43, step0=d,
                                                                                  trace=b),
                                     C, learned_steps, min(chunk, learned_steps), dev)
        found, med = hits(ltrace)
        return {"steps": learned_steps, "gpu_s": ltimes[-1][1], "chains_at_s": found, "median_first_step": med}

    # (a) the flip chains' own states, thinned to 10^5
    flat = ptrace[plain_steps // 2:].reshape(-1)
    pick = np.random.default_rng(7).choice(flat.size, size=train_samples, replace=False)
    data_a = torch.from_numpy(flat[pick].view(np.int64)).to(dev)
    net_a, t_a = train(data_a)
    res_a = learned(net_a)
    res_a.update({"training": "10^5 states of the flip chains", "train_gpu_s": t_a})
    net_a.close()
    # (b) exact samples of the chain-rule marginal sampler
    work = (lrstab.Simulator(n, local), lrstab.Simulator(n, local))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    samples = []
    for i in range(exact_samples):
        bits, _ = sim.marginal_sample(list(range(n)), L, K, seed=100 + i, work=work)
        samples.append(sum(int(b_) << q for q, b_ in enumerate(bits)))
    torch.cuda.synchronize()
    t_marg = time.perf_counter() - t0
    for w_ in work:
        w_.close()
    data_b = torch.tensor(samples, dtype=torch.int64, device=dev).repeat(train_samples // exact_samples + 1)
    data_b = data_b[:train_samples].contiguous()
    net_b, t_b = train(data_b)
    res_b = learned(net_b)
    res_b.update({"training": f"{exact_samples} chain-rule samples, replicated", "train_gpu_s": t_b,
                  "sampler_s": t_marg, "samples_are_the_shift": all(np.uint64(v) == s for v in samples)})
    net_b.close()
    sim.close()
    return {"workload": f"{cfg['name']}_chi{chi}", "chains": C, "chains_started_at_s": start_at_s,
            "flip": plain, "learned_on_flip_chains": res_a, "learned_on_exact_samples": res_b}


def hs_marginals_table_study(local=0, L=256, K=3, seed=0):
    """The paper's single-qubit marginal workload (end of Sec. 4.3, its table of norm
    estimation times): the 40-qubit hidden shift with 2, 4 and 6 CCZ, each CCZ in the
    8-term form (xi = 16/9) and the decomposition sparsified to chi = 39, 149 and 497
    terms (the state counts that table lists; delta = ||c||_1 / sqrt(chi) = 0.28, 0.26,
    0.25); for every one of the 40 qubits P(x_i = 1) from two median-of-means norm
    estimates of the projected decomposition (L K equatorial states each).  Reported:
    GPU wall seconds for all 40 marginals, the largest |P(x_i = 1) - s_i| (the
    infinity-norm error of the paper's figure), and the paper's single-threaded CPU
    time for the same shapes (context: other hardware)."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    n = 40
    paper_s = {2: 0.30, 4: 1.02, 6: 3.82}
    out = []
    for n_ccz, chi in ((2, 39), (4, 149), (6, 497)):
        ops, s = workloads.hidden_shift_circuit(n, n_ccz, workloads.SEED_BASE + 3)
        low = lrstab.lower_circuit(n, ops, "sum8")
        sim = lrstab.Simulator(n, local)
        sim.init_terms(low, chi, mode="sparsify", seed=90 + n_ccz)
        sim.apply_clifford(low.gates)
        work = (lrstab.Simulator(n, local), lrstab.Simulator(n, local))
        sim.marginal_sample([0], L, K, seed=seed, work=work)          # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p1 = []
        for q in range(n):
            _, probs = sim.marginal_sample([q], L, K, seed=seed + 1 + q, work=work)
            p0_, p1_ = probs[0]
            p1.append(p1_ / (p0_ + p1_) if p0_ + p1_ > 0 else 0.5)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        bits = np.array([(s >> q) & 1 for q in range(n)], np.float64)
        err = float(np.max(np.abs(np.array(p1) - bits)))
        delta = low.l1_norm / math.sqrt(chi)
        for w_ in (sim,) + work:
            w_.close()
        out.append({"ccz": n_ccz, "chi": chi, "delta": delta, "L": L, "K": K, "seconds_40_marginals": dt,
                    "ms_per_marginal": 1e3 * dt / n, "max_marginal_error": err,
                    "paper_cpu_seconds_per_norm_estimation": paper_s[n_ccz]})
    return {"workload": "hidden_shift_n40_single_qubit_marginals", "rows": out}


def marginal_study(local=0, w=8, L=256, K=3):
    """Chain-rule sampling of w bits by norm estimation (end of Sec. 4.3) on the n=40
    hidden shift (exact 2^16-term decomposition of |s>): every bit must come out as
    the shift's bit.  Each bit takes two median-of-means estimates (L K equatorial
    states each, the same states for both branches) of the projected decomposition."""
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    cfg = workloads.config_hidden_shift()
    n, chi = cfg["n"], cfg["chi"]
    low = lrstab.lower_circuit(n, cfg["ops"])
    sim = lrstab.Simulator(n, local)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    work = (lrstab.Simulator(n, local), lrstab.Simulator(n, local))
    qubits = list(range(0, n, n // w))[:w]
    sim.marginal_sample(qubits[:1], L, K, seed=1, work=work)      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bits, probs = sim.marginal_sample(qubits, L, K, seed=2, work=work)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ok = all(b == (cfg["shift"] >> q) & 1 for q, b in zip(qubits, bits))
    units = 2.0 * w * L * K * chi
    for s_ in (sim,) + work:
        s_.close()
    return {"workload": f"{cfg['name']}_w{w}", "w": w, "L": L, "K": K, "seconds": dt,
            "bits_per_s": w / dt, "A_term_per_s": units / dt, "bits_are_the_shift": ok,
            "max_wrong_branch_p": max(min(p) for p in probs)}


def mlp_gemm_study(local=0, n=64, H=2048, batch=16384, reps=5, bf16_peak=None):
    """Tensor-core throughput of the learned proposal's products: forward pass and
    one AdamW training step of the MADE network (n=64, H=2048, 16384 rows), with the
    tcgen05 GEMM and with the mma.sync GEMM.  FLOPs count the padded products
    (input width 64): forward 2 B (64 H + H^2 + 64 H), backward 2 B (2 * 64 H +
    2 H^2 + 64 H)."""
    import numpy as np
    import torch
    from paper_1808_00128_gb300 import lrstab, workloads
    dev = torch.device(f"cuda:{local}")
    net = lrstab.MLP(n, H, local)
    rng = np.random.default_rng(9)
    lim1, lim2 = 1 / np.sqrt(n), 1 / np.sqrt(H)
    net.set_params(dict(W1=rng.uniform(-lim1, lim1, (H, n)), b1=rng.uniform(-lim1, lim1, H),
                        W2=rng.uniform(-lim2, lim2, (H, H)), b2=rng.uniform(-lim2, lim2, H),
                        W3=rng.uniform(-lim2, lim2, (n, H)), b3=rng.uniform(-lim2, lim2, n)))
    x = torch.from_numpy(workloads.random_bitstrings(n, batch, workloads.SEED_BASE + 51).view(np.int64)).to(dev)
    logits = torch.empty((batch, n), dtype=torch.float32, device=dev)
    f_fwd = 2.0 * batch * (64 * H + H * H + H * 64)
    f_train = f_fwd + 2.0 * batch * (2 * 64 * H + 2 * H * H + 64 * H)
    res = {"n": n, "hidden": H, "batch": batch, "gflop_forward": f_fwd / 1e9, "gflop_train_step": f_train / 1e9}
    for name, kind in (("tcgen05", lrstab.MLP.GEMM_TCGEN05), ("mma_sync", lrstab.MLP.GEMM_MMA_SYNC)):
        net.gemm = kind
        row = {}
        for what, fn, fl in (("forward", lambda: net.forward(x), f_fwd),
                             ("train_step", lambda: net.train_step(x, lr=0.0), f_train)):
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                a, b = _ev()
                a.record()
                fn()
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            t = min(ts) * 1e-3
            row[what] = {"ms": t * 1e3, "tflops": fl / t / 1e12,
                         "frac_of_bf16_peak": fl / t / 1e12 / bf16_peak if bf16_peak else None}
        res[name] = row
    net.get_params()   # synchronises; reports a tcgen05 completion wait that gave up
    res["speedup_forward"] = res["mma_sync"]["forward"]["ms"] / res["tcgen05"]["forward"]["ms"]
    net.close()
    return res


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def side_step_study(name, local, alu_peak, hbm_peak, steps=5, warmup=3, certificate=False):
    """The same step on another workload (n = 40 random Clifford+T at chi = 2^16, or
    the paper's beta = pi/4 QAOA line): phase times, rooflines on both counts, the
    stated error bound, and optionally the sparsification certificate."""
    import torch
    from paper_1808_00128_gb300 import lrstab
    r = StepRunner(name, local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=r.dev)
    for w in range(warmup):
        r.step(idx=w)
    tuned = r.tune()
    r.step(idx=warmup)
    step_ms, phase_ms = r.timed(steps, warmup + 1, flush)
    ms = statistics.mean(step_ms)
    out = {"workload": r.cfg["name"], "n": r.n, "chi": r.chi, **r.shape, "ms_per_step": ms,
           "value": r.units() / (ms * 1e-3), "unit": UNIT, "tuned": tuned,
           "phases": r.rooflines(phase_ms, alu_peak, hbm_peak), "amplitude_error": r.error_statement()}
    if certificate:
        out["sparsification_certificate"] = lrstab.sparsification_certificate(r.sim, r.shape["L"], 3, seed=777)
        out["l1_norm"] = r.low.l1_norm
    r.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    peaks = _peaks()
    if args.mlp_gemm_only:
        print(json.dumps(mlp_gemm_study(0, reps=2, bf16_peak=peaks.get("bf16_tflops"))))
        return
    if args.hs_marginals:
        print(json.dumps(hs_marginals_table_study(0)))
        return
    if args.hidden_shift_chains:
        print(json.dumps(hidden_shift_chain_study(0)))
        return
    if args.hs_sum8_chains:
        print(json.dumps(hidden_shift_sum8_chain_study(0)))
        return
    if args.config5_graph:
        print(json.dumps(config5_graph_study(0)))
        return
    if args.qaoa_apply_only:
        print(json.dumps(qaoa_apply_only(0)))
        return
    if args.metropolis_only:
        print(json.dumps(metropolis_only(0, workload=args.workload)))
        return
    import torch
    from paper_1808_00128_gb300 import lrstab, sharding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    small = args.small
    if small:
        args.no_cpu_baseline = args.no_e2e = args.no_extra = args.no_sampler_study = True
    if world > 1:
        # the side studies are single-GPU measurements: a scaling run holds all its GPUs
        # only for the step itself
        args.no_extra = args.no_sampler_study = True
    # the oracle's host pool starts (spawn) before the first GPU call
    timer = OracleTimer() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lrstab.lib()

    r = StepRunner(args.workload, local, rank, small=small)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for w in range(args.warmup):
        r.step(idx=w)
    torch.cuda.synchronize()
    tuned = r.tune(cache_path=os.environ.get("LRS_TUNE_CACHE"))
    r.step(idx=args.warmup)
    torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        step_ms, phase_ms = r.timed(args.steps, args.warmup + 1, flush, world)
    ms = sharding.max_over_ranks(statistics.mean(step_ms), device=dev)
    units = r.units()
    value = world * units / (ms * 1e-3)

    hbm = peaks.get("hbm_gbs", 6800.0)
    alu = lrstab.alu_probe(local, 4000)
    rows = r.rooflines(phase_ms, alu, hbm)
    dom = max(("apply_clifford", "amplitude", "norm_estimate", "metropolis"), key=lambda p: phase_ms[p])
    roof = {k: v for k, v in rows[dom].items() if k not in ("ms", "rate", "rate_unit", "ms_per_metropolis_step")}
    roof["kernel"] = dom
    unit_count = {"norm_estimate": r.chi * r.shape["L"], "amplitude": r.chi * r.shape["B"],
                  "apply_clifford": r.chi, "metropolis": r.chi * r.shape["C"] * r.shape["T"]}[dom]
    roof["traffic"], roof["traffic_source"] = (None, None) if small else traffic_for(dom, unit_count)
    roof["peak_source"] = ("measured LOP3 probe on this GPU (of measured)" if roof["bound"] == "alu"
                           else "MEASURED_PEAKS.json hbm_gbs (of measured)")
    err = r.error_statement()
    cert = None if small else lrstab.sparsification_certificate(r.sim, r.shape["L"], 3, seed=777)

    e2e = None
    if not args.no_e2e:
        e_ms, h2d, d2h = r.e2e(args.steps, 100, flush)
        e_ms = sharding.max_over_ranks(e_ms, device=dev)
        e2e = {"value": world * units / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    r.close()

    cpu = cpu_py = parity = None
    if timer is not None:
        t0 = time.perf_counter()
        ct = COracleTimer(args.workload)
        k, n_x, n_a = 8192, 256, 8
        rates = ct.sample(k=k, n_x=n_x, n_a=n_a, alpha0=0)
        cpu = {"value": units / oracle_step_seconds(r.chi, r.shape, rates), "unit": UNIT,
               "cores": ct.threads, "kind": "oracle",
               "sample": f"{k} terms of the {r.cfg['name']} decomposition built by the C restatement of the "
                         f"oracle on {ct.threads} host threads, with {n_x} amplitude evaluations and {n_a} "
                         "equatorial inner products per term (exact integer sums); wall times per unit "
                         "scaled to one full step",
               "seconds": round(time.perf_counter() - t0, 1)}
        t0 = time.perf_counter()
        k, n_x, n_a = (16, 512, 4) if args.workload == "qaoa" else (24, 256, 8)
        rates = timer.sample(args.workload, k=k, n_x=n_x, n_a=n_a, alpha0=0)
        cpu_py = {"value": units / oracle_step_seconds(r.chi, r.shape, rates), "unit": UNIT,
                  "cores": timer.workers, "kind": "oracle (Python)",
                  "sample": f"{k} terms per core built by the Python oracle, {n_x} amplitude evaluations and "
                            f"{n_a} equatorial inner products per term; per-unit times scaled to one full step "
                            f"and divided by the parallelism achieved ({rates['parallel']:.1f} of "
                            f"{timer.workers} cores)",
                  "seconds": round(time.perf_counter() - t0, 1)}
        parity = [slice_parity(args.workload, local, timer=timer)]
    ess = side = None
    extra = {}
    if rank == 0 and not args.no_sampler_study:
        ess = {"n20_exact_reference": sampler_study(local),
               "n50_qaoa_instance": sampler_study(local, chi=1 << 18, qaoa_instance=True, plain_steps=600,
                                                  learned_steps=100, ref_steps=1200, burn=100)}
    if rank == 0 and not args.no_extra:
        other = "mid" if args.workload == "qaoa" else "qaoa"
        side = side_step_study(other, local, alu, hbm)
        if timer is not None:
            parity.append(slice_parity(other, local, timer=timer))
        try:
            c5 = config5_graph_study(local)
        except Exception as e:   # reported in the line; the step's numbers above stand
            c5 = {"error": str(e)[:300]}
        extra = {"batch8": batch_study(local), "config5_graph": c5,
                 "mlp_gemm": mlp_gemm_study(local, bf16_peak=peaks.get("bf16_tflops")),
                 "marginals": marginal_study(local), "gadget_vs_sum": gadget_study(local),
                 "prefix_sharing": prefix_study(local), "hidden_shift_sum8": hidden_shift_sum8_study(local),
                 "hidden_shift_chains": hidden_shift_chain_study(local),
                 "hs_marginals_table": hs_marginals_table_study(local)}
        if args.workload == "qaoa":
            extra["qaoa_beta_pi4"] = side_step_study("qaoa_pi4", local, alu, hbm, certificate=True)
    if timer is not None:
        timer.close()
    if rank != 0:
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64+f32", "data": "synthetic",
           "config": {"workload": r.cfg["name"] + (f"_chi{r.chi}" if small else ""), "n": r.n, "chi": r.chi,
                      "batch": r.shape["B"], "L": r.shape["L"], "chains": r.shape["C"],
                      "metropolis_steps": r.shape["T"], "gates": len(r.low.gates), "slots": len(r.low.slots),
                      "l2": "flushed (256 MB write) before every timed step",
                      "parallelism": f"replicas x{world}", "tuned": tuned},
           "roofline": roof, "phases": rows, "amplitude_error": err, "parity_slices": parity,
           "sparsification_certificate": cert,
           "cpu_baseline": cpu, "cpu_baseline_python": cpu_py, "e2e": e2e, "gpu_launches": launches_per_step(r.shape["T"], r.lookahead) * args.steps,
           "clocks": clk.summary(), "ess": ess, "side_step": side, **extra}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
