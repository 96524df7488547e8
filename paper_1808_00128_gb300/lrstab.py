"""ctypes binding of liblrstab.so (argument marshalling only).

Every computation happens in the CUDA library; this module converts Python
circuits and torch tensors into the C ABI's plain pointers and sizes.  There
is no CPU fallback: if the library is missing or a call fails, it raises.

Device buffers are torch tensors on the context's device (PyTorch serves as
the device allocator and stream provider).  Basis strings are 64-bit words
(torch.int64 or torch.uint64 tensors) holding qubit j in bit j.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrstab.so")

# ---- C enums (include/lrstab.h) ----------------------------------------------------
OP = dict(H=0, S=1, SDG=2, Z=3, CX=4, CZ=5, P0=6, P1=7, SLOT=8)
CKIND = dict(H=0, S=1, SDG=2, Z=3, CX=4, CZ=5, T=6, RZ=7, CCZ=8)
CCZ_MODE = dict(proj=0, sum8=1)
TUNE = dict(amp_blocks_per_sm=0, norm_max_tiles=1, mc_chains_per_block=2, norm_max_folds=3, mc_stages=4,
            apply_lanes=5, norm_fuse_folds=6, mc_lookahead=7)
MODE = dict(exact=0, sparsify=1)
STATUS = {0: "LRS_OK", -1: "LRS_ERR_ARG", -2: "LRS_ERR_OOM", -3: "LRS_ERR_CUDA",
          -4: "LRS_ERR_TIMEOUT", -5: "LRS_ERR_STATE", -6: "LRS_ERR_UNSUPPORTED"}

GATE_DT = np.dtype([("op", "u1"), ("q", "u1"), ("r", "<u2")])
SLOT_DT = np.dtype([("n_choices", "<i4"), ("k_off", "<i4", (8,)), ("k_len", "<i4", (8,)),
                    ("c_re", "<f8", (8,)), ("c_im", "<f8", (8,))], align=True)
COP_DT = np.dtype([("kind", "<i4"), ("q", "<i4", (3,)), ("theta", "<f8")], align=True)

EXPORTED = ["lrs_lower_circuit", "lrs_create", "lrs_destroy", "lrs_last_error", "lrs_init_terms", "lrs_reinit_terms",
            "lrs_apply_clifford", "lrs_amplitude", "lrs_norm_estimate", "lrs_sample_terms",
            "lrs_chains_init", "lrs_metropolis_step", "lrs_export_terms", "lrs_info",
            "lrs_alu_probe", "lrs_amplitude_noalloc", "lrs_mlp_create", "lrs_mlp_destroy",
            "lrs_mlp_info", "lrs_mlp_set_gemm", "lrs_mlp_get_gemm", "lrs_mlp_set_params", "lrs_mlp_get_params", "lrs_mlp_forward",
            "lrs_mlp_backward", "lrs_mlp_train_step", "lrs_mlp_sample", "lrs_metropolis_learned",
            "lrs_apply_clifford_batch", "lrs_set_tuning", "lrs_get_tuning", "lrs_copy_terms",
            "lrs_norm_median_of_means", "lrs_marginal_sample", "lrs_lower_gadget",
            "lrs_apply_circuit_shared", "lrs_decomposition_stats", "lrs_sparsification_certificate",
            "lrs_debug_inject_wait_timeout", "lrs_mlp_debug_inject_wait_timeout", "lrs_chains_set_amplitude",
            "lrs_metropolis_propose", "lrs_metropolis_accept", "lrs_norm_overlaps",
            "lrs_norm_eta_from_overlaps", "lrs_amplitude_batch"]


class LrsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load liblrstab.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, u64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
    L.lrs_last_error.restype = C.c_char_p
    sigs = {
        "lrs_lower_circuit": [i32, vp, i64, i32, vp, i64, vp, vp, i64, vp, vp, i64, vp],
        "lrs_create": [i32, i32, vp, vp],
        "lrs_destroy": [vp],
        "lrs_init_terms": [vp, vp, i64, vp, i64, i64, i64, i64, i32, u64, vp],
        "lrs_apply_clifford": [vp, vp, i64, vp],
        "lrs_amplitude": [vp, vp, i64, vp, vp, vp],
        "lrs_norm_estimate": [vp, i64, u64, vp, vp, vp],
        "lrs_sample_terms": [vp, i64, u64, vp, vp, vp],
        "lrs_chains_init": [vp, i64, vp, vp],
        "lrs_metropolis_step": [vp, i64, u64, i64, vp, vp, vp, vp],
        "lrs_export_terms": [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "lrs_info": [vp, vp, vp, vp],
        "lrs_alu_probe": [i32, i64, vp],
        "lrs_amplitude_noalloc": [vp, vp, i64, vp, vp],
        "lrs_mlp_create": [i32, i32, i32, vp],
        "lrs_mlp_destroy": [vp],
        "lrs_mlp_info": [vp, vp, vp, vp],
        "lrs_mlp_set_gemm": [vp, i32],
        "lrs_mlp_get_gemm": [vp, vp],
        "lrs_mlp_set_params": [vp, vp],
        "lrs_mlp_get_params": [vp, vp, vp],
        "lrs_mlp_forward": [vp, vp, i64, vp, vp, vp],
        "lrs_mlp_backward": [vp, vp, i64, vp, vp],
        "lrs_mlp_train_step": [vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, vp, vp],
        "lrs_mlp_sample": [vp, i64, u64, i64, vp, vp, vp],
        "lrs_metropolis_learned": [vp, vp, i64, u64, i64, vp, vp, vp, vp, vp],
        "lrs_apply_clifford_batch": [vp, vp, vp, i32, vp],
        "lrs_set_tuning": [vp, i32, i64],
        "lrs_copy_terms": [vp, vp, vp],
        "lrs_reinit_terms": [vp, u64, vp],
        "lrs_apply_circuit_shared": [vp, vp, i64, vp],
        "lrs_lower_gadget": [i32, vp, i64, i32, vp, vp, i64, vp, vp, i64, vp, vp, i64, vp],
        "lrs_norm_median_of_means": [vp, i64, i32, u64, vp, vp],
        "lrs_marginal_sample": [vp, vp, vp, vp, i32, i64, i32, u64, vp, vp, vp],
        "lrs_get_tuning": [vp, i32, vp],
        "lrs_decomposition_stats": [vp, i64, vp, vp, vp],
        "lrs_sparsification_certificate": [vp, i64, i32, u64, vp, vp],
        "lrs_debug_inject_wait_timeout": [vp],
        "lrs_mlp_debug_inject_wait_timeout": [vp],
        "lrs_chains_set_amplitude": [vp, vp, vp],
        "lrs_metropolis_propose": [vp, u64, i64, vp, vp],
        "lrs_metropolis_accept": [vp, vp, u64, i64, vp, vp],
        "lrs_norm_overlaps": [vp, i64, u64, vp, vp],
        "lrs_norm_eta_from_overlaps": [vp, i64, vp, vp, vp],
        "lrs_amplitude_batch": [vp, vp, vp, vp, i32, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise LrsError(rc, lib().lrs_last_error().decode())


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- circuits ------------------------------------------------------------------------
def circuit_ops(ops) -> np.ndarray:
    """Workload tuples ('H', q), ('CX', c, t), ('RZ', q, theta), ... -> lrs_circuit_op[]."""
    arr = np.zeros(len(ops), dtype=COP_DT)
    for i, op in enumerate(ops):
        name = op[0]
        arr[i]["kind"] = CKIND[name]
        if name == "RZ":
            arr[i]["q"][0] = op[1]
            arr[i]["theta"] = op[2]
        else:
            for t, q in enumerate(op[1:]):
                arr[i]["q"][t] = q
    return arr


CERT_DT = np.dtype([("omega_norm2", "<f8"), ("stderr_mean", "<f8"), ("delta2", "<f8"), ("bound", "<f8"),
                    ("bound_upper", "<f8"), ("conclusive", "<i4"), ("reserved", "<i4")])


class Lowered:
    """Lowered circuit: gates (with SLOT entries), slot tables and K_j gate lists, on
    n_total qubits (the circuit's own n, or n + tau for the gadget form)."""

    def __init__(self, gates, slots, kgates, n_total=None):
        self.gates, self.slots, self.kgates = gates, slots, kgates
        self.n_total = n_total

    def _stats(self):
        l1, chi, lg = C.c_double(0.0), C.c_int64(0), C.c_double(0.0)
        slots = np.ascontiguousarray(self.slots)
        _check(lib().lrs_decomposition_stats(_ptr(slots), len(slots), C.byref(l1), C.byref(chi), C.byref(lg)))
        return l1.value, chi.value, lg.value

    @property
    def exact_chi(self) -> int:
        """Terms of the exact enumeration (lrs_decomposition_stats; -1 above 2^62)."""
        return self._stats()[1]

    @property
    def l1_norm(self) -> float:
        """||c||_1 of the whole decomposition (lrs_decomposition_stats)."""
        return self._stats()[0]


def sparsification_certificate(sim: "Simulator", L: int, K: int, seed: int, stream=None) -> dict:
    """lrs_sparsification_certificate: Lemma (Sparsification tail bound) for the
    sparsified state held by `sim`."""
    out = np.zeros(1, CERT_DT)
    _check(lib().lrs_sparsification_certificate(sim._h, L, K, seed & (2 ** 64 - 1), _ptr(out), _stream(stream)))
    r = {k: float(out[0][k]) for k in ("omega_norm2", "stderr_mean", "delta2", "bound", "bound_upper")}
    r.update(conclusive=bool(out[0]["conclusive"]), L=L, K=K)
    return r


def lower_circuit(n: int, ops, ccz_mode: str = "proj", method: str = "sum") -> Lowered:
    """lrs_lower_circuit (method "sum": sum-over-Cliffords slots on n qubits) or
    lrs_lower_gadget (method "gadget": fixed-sample gadgets on n + tau qubits)."""
    cops = circuit_ops(ops)
    ng, ns, nk, nt = C.c_int64(0), C.c_int64(0), C.c_int64(0), C.c_int32(n)
    gates = np.zeros(max(1, 8 * len(ops) + 8), GATE_DT)
    slots = np.zeros(max(1, len(ops)), SLOT_DT)
    kg = np.zeros(max(1, 8 * len(ops)), GATE_DT)
    if method == "gadget":
        rc = lib().lrs_lower_gadget(n, _ptr(cops), len(ops), CCZ_MODE[ccz_mode], C.byref(nt), _ptr(gates),
                                    len(gates), C.byref(ng), _ptr(slots), len(slots), C.byref(ns), _ptr(kg),
                                    len(kg), C.byref(nk))
    elif method == "sum":
        rc = lib().lrs_lower_circuit(n, _ptr(cops), len(ops), CCZ_MODE[ccz_mode], _ptr(gates), len(gates),
                                     C.byref(ng), _ptr(slots), len(slots), C.byref(ns), _ptr(kg), len(kg),
                                     C.byref(nk))
    else:
        raise ValueError(f"unknown lowering method {method!r}")
    _check(rc)
    return Lowered(gates[: ng.value].copy(), slots[: ns.value].copy(), kg[: nk.value].copy(), nt.value)


def gates_array(gates) -> np.ndarray:
    """('H', q) / ('CX', q, r) / ('P1', q) / ('SLOT', p) tuples -> lrs_gate[]."""
    arr = np.zeros(len(gates), GATE_DT)
    for i, g in enumerate(gates):
        arr[i]["op"] = OP[g[0]]
        if g[0] == "SLOT":
            arr[i]["r"] = g[1]
        else:
            arr[i]["q"] = g[1]
            if len(g) > 2:
                arr[i]["r"] = g[2]
    return arr


def alu_probe(device: int = 0, iters: int = 20000) -> float:
    """Sustained 32-bit LOP3 rate of the device (ops/s)."""
    out = C.c_double(0.0)
    _check(lib().lrs_alu_probe(device, iters, C.byref(out)))
    return out.value


# ---- simulator context ------------------------------------------------------------------
class LrsOptions(C.Structure):
    _fields_ = [("size", C.c_int32), ("tuning_mask", C.c_uint32), ("tuning", C.c_int64 * 16)]


def options(tuning: dict | None = None) -> LrsOptions:
    """lrs_options with the given initial launch knobs ({name: value}, names of TUNE)."""
    o = LrsOptions()
    o.size = C.sizeof(LrsOptions)
    for name, value in (tuning or {}).items():
        i = TUNE[name]
        o.tuning_mask |= 1 << i
        o.tuning[i] = int(value)
    return o


class Simulator:
    """One lrs_ctx: chi CH-form terms of an n-qubit circuit on one GPU.  `tuning`:
    initial launch knobs ({name: value}), passed to lrs_create as lrs_options."""

    def __init__(self, n: int, device: int = 0, tuning: dict | None = None):
        self.n = n
        self.device = device
        h = C.c_void_p()
        opts = options(tuning) if tuning else None
        _check(lib().lrs_create(device, n, C.byref(opts) if opts is not None else None, C.byref(h)))
        self._h = h
        self.chi = 0
        self.n_slots = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().lrs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def init_terms(self, lowered: Lowered, chi: int, mode: str = "sparsify", seed: int = 0,
                   alpha0: int = 0, chi_total: int | None = None, stream=None):
        """Terms alpha0 .. alpha0+chi-1 of a chi_total-term decomposition (default: all)."""
        chi_total = chi if chi_total is None else chi_total
        _check(lib().lrs_init_terms(self._h, _ptr(lowered.slots), len(lowered.slots),
                                    _ptr(lowered.kgates), len(lowered.kgates), chi_total, alpha0, chi,
                                    MODE[mode], seed & (2 ** 64 - 1), _stream(stream)))
        self.chi = chi
        self.alpha0 = alpha0
        self.chi_total = chi_total
        self.n_slots = len(lowered.slots)

    def reinit_terms(self, seed: int, stream=None):
        """The last init_terms again from the tables on the device (new sparsification
        seed); graph-capturable."""
        _check(lib().lrs_reinit_terms(self._h, seed & (2 ** 64 - 1), _stream(stream)))

    def apply_clifford(self, gates: np.ndarray, stream=None):
        _check(lib().lrs_apply_clifford(self._h, _ptr(gates), len(gates), _stream(stream)))

    def apply_circuit_shared(self, gates: np.ndarray, stream=None):
        """lrs_apply_circuit_shared: the lowered circuit on fresh exact-mode terms,
        sharing the work of common choice prefixes."""
        _check(lib().lrs_apply_circuit_shared(self._h, _ptr(gates), len(gates), _stream(stream)))

    def amplitude(self, x, out=None, err=None, stream=None):
        """x: int64/uint64 CUDA tensor [B] -> float64 CUDA tensor [B, 2] (Re, Im).
        err: optional float32 CUDA tensor [B] receiving the per-result error bound."""
        import torch
        if out is None:
            out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
        _check(lib().lrs_amplitude(self._h, _ptr(x), x.numel(), _ptr(out), _ptr(err), _stream(stream)))
        return out

    def amplitude_noalloc(self, x, out, stream=None):
        """As amplitude(), through the entry point that allocates no device memory
        (`out` must be supplied: float64 CUDA tensor [B, 2])."""
        _check(lib().lrs_amplitude_noalloc(self._h, _ptr(x), x.numel(), _ptr(out), _stream(stream)))
        return out

    def norm_estimate(self, L: int, seed: int, eta=None, want_mean: bool = False, stream=None):
        import torch
        if eta is None:
            eta = torch.empty(L, dtype=torch.float64, device=f"cuda:{self.device}")
        mean = C.c_double(0.0)
        _check(lib().lrs_norm_estimate(self._h, L, seed & (2 ** 64 - 1), _ptr(eta),
                                       C.byref(mean) if want_mean else None, _stream(stream)))
        return (eta, mean.value) if want_mean else eta

    def norm_overlaps(self, L: int, seed: int, ov=None, stream=None):
        """lrs_norm_overlaps: 2^{n/2} <phi_{A_l}|psi> over this context's terms (float64
        CUDA tensor [L, 2])."""
        import torch
        if ov is None:
            ov = torch.empty((L, 2), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(lib().lrs_norm_overlaps(self._h, L, seed & (2 ** 64 - 1), _ptr(ov), _stream(stream)))
        return ov

    def norm_eta_from_overlaps(self, ov, eta=None, stream=None):
        """lrs_norm_eta_from_overlaps: eta_l = |ov_l|^2 of summed overlaps."""
        import torch
        L = ov.shape[0]
        if eta is None:
            eta = torch.empty(L, dtype=torch.float64, device=ov.device)
        _check(lib().lrs_norm_eta_from_overlaps(self._h, L, _ptr(ov), _ptr(eta), _stream(stream)))
        return eta

    def norm_median_of_means(self, L: int, K: int, seed: int, stream=None) -> float:
        est = C.c_double(0.0)
        _check(lib().lrs_norm_median_of_means(self._h, L, K, seed & (2 ** 64 - 1), C.byref(est),
                                              _stream(stream)))
        return est.value

    def copy_terms_from(self, src: "Simulator", stream=None):
        _check(lib().lrs_copy_terms(self._h, src._h, _stream(stream)))
        chi, ns = C.c_int64(0), C.c_int64(0)
        _check(lib().lrs_info(self._h, C.byref(chi), None, C.byref(ns)))
        self.chi, self.n_slots = chi.value, ns.value
        self.chi_total = getattr(src, "chi_total", chi.value)

    def marginal_sample(self, qubits, L: int, K: int, seed: int, work=None, stream=None):
        """Chain-rule sample of the bits on `qubits` (lrs_marginal_sample).  Returns
        (bits, probs) with probs[i] = (p0, p1) of step i.  `work`: two Simulators with
        the same n (created and closed here when None)."""
        own = work is None
        if own:
            work = (Simulator(self.n, self.device), Simulator(self.n, self.device))
        try:
            q = np.ascontiguousarray(qubits, dtype=np.int32)
            bits = np.zeros(len(q), np.uint8)
            probs = np.zeros((len(q), 2), np.float64)
            _check(lib().lrs_marginal_sample(self._h, work[0]._h, work[1]._h, _ptr(q), len(q), L, K,
                                             seed & (2 ** 64 - 1), _ptr(bits), _ptr(probs), _stream(stream)))
        finally:
            if own:
                work[0].close()
                work[1].close()
        return bits.tolist(), [tuple(p) for p in probs]

    def sample_terms(self, count: int, seed: int, x=None, alpha=None, stream=None):
        import torch
        if x is None:
            x = torch.empty(count, dtype=torch.int64, device=f"cuda:{self.device}")
        _check(lib().lrs_sample_terms(self._h, count, seed & (2 ** 64 - 1), _ptr(x), _ptr(alpha),
                                      _stream(stream)))
        return x

    def chains_init(self, x, stream=None):
        _check(lib().lrs_chains_init(self._h, x.numel(), _ptr(x), _stream(stream)))
        self._chains = x.numel()

    def metropolis(self, steps: int, seed: int, step0: int = 0, x_out=None, p_out=None, trace=None,
                   stream=None):
        _check(lib().lrs_metropolis_step(self._h, steps, seed & (2 ** 64 - 1), step0, _ptr(x_out),
                                         _ptr(p_out), _ptr(trace), _stream(stream)))

    def chains_set_amplitude(self, amp, stream=None):
        """lrs_chains_set_amplitude: P(x_c) from summed amplitudes (float64 [C, 2])."""
        _check(lib().lrs_chains_set_amplitude(self._h, _ptr(amp), _stream(stream)))

    def metropolis_propose(self, seed: int, step: int, amp=None, stream=None):
        """lrs_metropolis_propose: this shard's partial amplitudes of the proposals of
        step `step` (float64 CUDA tensor [C, 2])."""
        import torch
        if amp is None:
            amp = torch.empty((self._chains, 2), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(lib().lrs_metropolis_propose(self._h, seed & (2 ** 64 - 1), step, _ptr(amp), _stream(stream)))
        return amp

    def metropolis_accept(self, amp, seed: int, step: int, trace=None, stream=None):
        """lrs_metropolis_accept on the summed amplitudes of step `step`."""
        _check(lib().lrs_metropolis_accept(self._h, _ptr(amp), seed & (2 ** 64 - 1), step, _ptr(trace),
                                           _stream(stream)))

    def set_tuning(self, name: str, value: int):
        _check(lib().lrs_set_tuning(self._h, TUNE[name], int(value)))

    def get_tuning(self, name: str) -> int:
        v = C.c_int64(0)
        _check(lib().lrs_get_tuning(self._h, TUNE[name], C.byref(v)))
        return v.value

    def debug_inject_wait_timeout(self):
        """lrs_debug_inject_wait_timeout (failure-path tests)."""
        _check(lib().lrs_debug_inject_wait_timeout(self._h))

    def export_terms(self, first: int = 0, count: int | None = None) -> dict:
        count = self.chi - first if count is None else count
        n, ns = self.n, self.n_slots
        out = dict(F=np.zeros((count, n), np.uint64), G=np.zeros((count, n), np.uint64),
                   M=np.zeros((count, n), np.uint64), gamma=np.zeros((count, n), np.uint8),
                   v=np.zeros(count, np.uint64), s=np.zeros(count, np.uint64),
                   omega=np.zeros(count, np.int32), coef=np.zeros((count, 2), np.float32),
                   choice=np.zeros((count, max(ns, 1)), np.uint8))
        _check(lib().lrs_export_terms(self._h, first, count, *[_ptr(out[k]) for k in
                                      ("F", "G", "M", "gamma", "v", "s", "omega", "coef", "choice")]))
        return out


# ---- learned proposal ---------------------------------------------------------------------
class MLP:
    """MADE proposal network (lrs_mlp) on one GPU."""

    def __init__(self, n: int, hidden: int = 512, device: int = 0):
        self.n, self.hidden, self.device = n, hidden, device
        h = C.c_void_p()
        _check(lib().lrs_mlp_create(device, n, hidden, C.byref(h)))
        self._h = h
        npar = C.c_int64(0)
        _check(lib().lrs_mlp_info(h, None, None, C.byref(npar)))
        self.n_params = npar.value

    def close(self):
        if getattr(self, "_h", None):
            lib().lrs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    GEMM_TCGEN05, GEMM_MMA_SYNC = 0, 1

    @property
    def gemm(self) -> int:
        k = C.c_int32(0)
        _check(lib().lrs_mlp_get_gemm(self._h, C.byref(k)))
        return k.value

    @gemm.setter
    def gemm(self, kind: int):
        _check(lib().lrs_mlp_set_gemm(self._h, kind))

    def pack(self, params: dict) -> np.ndarray:
        return np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    def unpack(self, flat: np.ndarray) -> dict:
        n, H = self.n, self.hidden
        shapes = dict(W1=(H, n), b1=(H,), W2=(H, H), b2=(H,), W3=(n, H), b3=(n,))
        out, o = {}, 0
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            sz = int(np.prod(shapes[k]))
            out[k] = flat[o:o + sz].reshape(shapes[k])
            o += sz
        return out

    def debug_inject_wait_timeout(self):
        """lrs_mlp_debug_inject_wait_timeout (failure-path tests)."""
        _check(lib().lrs_mlp_debug_inject_wait_timeout(self._h))

    def set_params(self, params: dict):
        flat = np.ascontiguousarray(self.pack(params))
        _check(lib().lrs_mlp_set_params(self._h, _ptr(flat)))

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        g = np.zeros(self.n_params, np.float32)
        _check(lib().lrs_mlp_get_params(self._h, _ptr(p), _ptr(g)))
        return self.unpack(p), self.unpack(g)

    def forward(self, x, stream=None):
        import torch
        logits = torch.empty((x.numel(), self.n), dtype=torch.float32, device=x.device)
        logq = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
        _check(lib().lrs_mlp_forward(self._h, _ptr(x), x.numel(), _ptr(logits), _ptr(logq),
                                     _stream(stream)))
        return logits, logq

    def backward(self, x, stream=None):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(lib().lrs_mlp_backward(self._h, _ptr(x), x.numel(), _ptr(loss), _stream(stream)))
        return loss

    def train_step(self, x, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, loss=None,
                   stream=None):
        _check(lib().lrs_mlp_train_step(self._h, _ptr(x), x.numel(), lr, beta1, beta2, eps, wd,
                                        _ptr(loss), _stream(stream)))

    def sample(self, count: int, seed: int, sample0: int = 0, stream=None):
        import torch
        y = torch.empty(count, dtype=torch.int64, device=f"cuda:{self.device}")
        lq = torch.empty(count, dtype=torch.float32, device=f"cuda:{self.device}")
        _check(lib().lrs_mlp_sample(self._h, count, seed & (2 ** 64 - 1), sample0, _ptr(y), _ptr(lq),
                                    _stream(stream)))
        return y, lq


def metropolis_learned(sim: "Simulator", mlp: MLP, steps: int, seed: int, step0: int = 0,
                       x_out=None, p_out=None, trace=None, accepts=None, stream=None):
    _check(lib().lrs_metropolis_learned(sim._h, mlp._h, steps, seed & (2 ** 64 - 1), step0,
                                        _ptr(x_out), _ptr(p_out), _ptr(trace), _ptr(accepts),
                                        _stream(stream)))


def amplitude_batch(sims, xs, outs=None, stream=None):
    """lrs_amplitude_batch: <x|psi> of several circuits (same width, one device) in one
    amplitude launch and one reduction; returns float64 CUDA tensors [B_i, 2]."""
    import torch
    k = len(sims)
    if outs is None:
        outs = [torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device) for x in xs]
    handles = (C.c_void_p * k)(*[s._h.value for s in sims])
    xp = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
    bs = (C.c_int64 * k)(*[x.numel() for x in xs])
    op = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
    _check(lib().lrs_amplitude_batch(handles, xp, bs, op, k, _stream(stream)))
    return outs


def apply_clifford_batch(sims, gate_lists, stream=None):
    """One launch pushing each Simulator's terms through its gate list."""
    k = len(sims)
    handles = (C.c_void_p * k)(*[s._h.value for s in sims])
    garrs = [np.ascontiguousarray(g) for g in gate_lists]
    ptrs = (C.c_void_p * k)(*[g.ctypes.data for g in garrs])
    counts = (C.c_int64 * k)(*[len(g) for g in garrs])
    _check(lib().lrs_apply_clifford_batch(handles, ptrs, counts, k, _stream(stream)))
