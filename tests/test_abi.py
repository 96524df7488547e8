"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/lrstab.h declares; the host lowering of
non-Clifford gates matches the oracle's decomposition tables; calls that need
a device fail with an error code instead of crashing."""
import os
import re

import numpy as np
import pytest

from oracle import decomp
from paper_1808_00128_gb300 import _build, lrstab, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lrstab.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lrstab.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"(?:lrs_status|const char\s*\*)\s*(lrs_\w+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lrstab.EXPORTED)


def test_struct_layouts():
    assert lrstab.GATE_DT.itemsize == 4
    assert lrstab.SLOT_DT.itemsize == 200
    assert lrstab.COP_DT.itemsize == 24


@pytest.mark.parametrize("ccz_mode", ["proj", "sum8"])
@pytest.mark.parametrize("method", ["sum", "gadget"])
def test_lowering_matches_oracle_tables(lib, ccz_mode, method):
    ops = workloads.random_clifford_t(7, 60, 5, seed=3)
    ops += [("RZ", 2, 0.3), ("RZ", 4, -0.7), ("CCZ", 1, 3, 5), ("SDG", 0), ("Z", 6)]
    low = lrstab.lower_circuit(7, ops, ccz_mode, method=method)
    if method == "gadget":
        n_total, gates, slots = decomp.lower_gadget(7, ops, ccz_mode)
        assert low.n_total == n_total == 7 + 5 + 2 + 3
    else:
        gates, slots = decomp.lower(ops, ccz_mode)
        assert low.n_total == 7
    assert len(low.gates) == len(gates)
    inv = {v: k for k, v in lrstab.OP.items()}
    for g, og in zip(low.gates, gates):
        name = inv[int(g["op"])]
        if name == "SLOT":
            assert og == ("SLOT", int(g["r"]))
        elif name in ("CX", "CZ"):
            assert og == (name, int(g["q"]), int(g["r"]))
        else:
            assert og == (name, int(g["q"]))
    assert len(low.slots) == len(slots)
    for s, dec in zip(low.slots, slots):
        assert s["n_choices"] == len(dec)
        for j, (c, kg) in enumerate(dec):
            assert complex(s["c_re"][j], s["c_im"][j]) == pytest.approx(c, abs=4e-15)
            sub = low.kgates[s["k_off"][j]: s["k_off"][j] + s["k_len"][j]]
            got = []
            for g in sub:
                nm = inv[int(g["op"])]
                got.append((nm, int(g["q"]), int(g["r"])) if nm in ("CX", "CZ") else (nm, int(g["q"])))
            assert got == kg


def test_lowering_rejects_bad_input(lib):
    with pytest.raises(lrstab.LrsError):
        lrstab.lower_circuit(3, [("CX", 1, 1)])
    with pytest.raises(lrstab.LrsError):
        lrstab.lower_circuit(3, [("H", 3)])
    with pytest.raises(lrstab.LrsError):
        lrstab.lower_circuit(65, [])
    with pytest.raises(lrstab.LrsError):      # 40 + 25 ancillas > 64 qubits
        lrstab.lower_circuit(40, [("T", q % 40) for q in range(25)], method="gadget")


def test_create_without_device_is_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(lrstab.LrsError):
        lrstab.Simulator(4, 0)
    with pytest.raises(lrstab.LrsError):
        lrstab.Simulator(0, 0)


def test_lowered_l1_norm_matches_oracle_tables():
    """||c||_1 of the lowered slots (the sparsification certificate's delta^2 =
    ||c||_1^2 / chi) equals the oracle's product of slot l1 norms."""
    from oracle import decomp
    for cfg in (workloads.config_tiny(), workloads.config_mid()):
        low = lrstab.lower_circuit(cfg["n"], cfg["ops"])
        _, slots = decomp.lower(cfg["ops"])
        assert low.l1_norm == pytest.approx(decomp.l1_norm(slots), rel=1e-12)


def test_decomposition_stats_match_oracle_tables(lib):
    """lrs_decomposition_stats: ||c||_1 and the exact term count of the lowered slot
    tables equal the oracle's, with -1 once the count exceeds 2^62."""
    import math
    for cfg in (workloads.config_tiny(), workloads.config_mid(), workloads.config_qaoa(),
                workloads.config_hidden_shift()):
        low = lrstab.lower_circuit(cfg["n"], cfg["ops"])
        _, slots = decomp.lower(cfg["ops"])
        l1, chi, lg = low._stats()
        assert l1 == pytest.approx(decomp.l1_norm(slots), rel=1e-12)
        want = decomp.exact_chi(slots)
        assert chi == (want if want <= 2 ** 62 else -1)
        assert lg == pytest.approx(math.log2(want), rel=1e-12)
