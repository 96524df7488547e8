"""Prefix-shared circuit application (lrs_apply_circuit_shared): the terms equal those
of the plain per-term application bit for bit (exact decompositions of the tiny
Clifford+T circuit, the full-size hidden shift, and the gadget form), and the call
refuses sparsified or already-evolved terms."""
import numpy as np
import pytest

from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu


def _both(n, ops, method="sum"):
    low = lrstab.lower_circuit(n, ops, method=method)
    chi = low.exact_chi
    a = lrstab.Simulator(low.n_total, 0)
    a.init_terms(low, chi, mode="exact")
    a.apply_clifford(low.gates)
    b = lrstab.Simulator(low.n_total, 0)
    b.init_terms(low, chi, mode="exact")
    b.apply_circuit_shared(low.gates)
    ea, eb = a.export_terms(), b.export_terms()
    for k in ea:
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    return a, b, low


@pytest.mark.parametrize("case", ["tiny", "hidden_shift", "tiny_gadget"])
def test_shared_prefixes_equal_plain_application(case):
    require_cuda()
    if case == "hidden_shift":
        cfg = workloads.config_hidden_shift()
        a, b, _ = _both(cfg["n"], cfg["ops"])
    else:
        cfg = workloads.config_tiny()
        a, b, _ = _both(cfg["n"], cfg["ops"], "gadget" if case == "tiny_gadget" else "sum")
    a.close()
    b.close()


def test_shared_application_refuses_other_terms():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops = cfg["n"], cfg["ops"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, 64, mode="sparsify", seed=1)
    with pytest.raises(lrstab.LrsError):
        sim.apply_circuit_shared(low.gates)                  # sparsified terms
    sim.init_terms(low, 64, mode="exact")
    sim.apply_clifford(low.gates[:3])
    with pytest.raises(lrstab.LrsError):
        sim.apply_circuit_shared(low.gates)                  # no longer fresh
    sim.init_terms(low, 64, mode="exact")
    gates = low.gates.copy()
    slot_rows = np.flatnonzero(gates["op"] == lrstab.OP["SLOT"])
    gates[slot_rows[0]], gates[slot_rows[1]] = gates[slot_rows[1]].copy(), gates[slot_rows[0]].copy()
    with pytest.raises(lrstab.LrsError):
        sim.apply_circuit_shared(gates)                      # slots out of order
    sim.close()
