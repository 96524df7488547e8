"""Closed-form constants printed in the paper, checked against the oracle."""
import json
import math
import os

import numpy as np
import pytest

from oracle import decomp, dense

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_stabilizer_fidelities():
    """F(T) = |<+|T>|^2 and F(CCZ) = |<+++|CCZ>|^2 (Sec. 2.4.2)."""
    plus1 = dense.run(1, [("H", 0)])
    t_state = dense.run(1, [("H", 0), ("T", 0)])
    assert abs(np.vdot(plus1, t_state)) ** 2 == pytest.approx(GOLD["F_T"], rel=1e-14)
    plus3 = dense.run(3, [("H", 0), ("H", 1), ("H", 2)])
    ccz = dense.run(3, [("H", 0), ("H", 1), ("H", 2), ("CCZ", 0, 1, 2)])
    assert abs(np.vdot(plus3, ccz)) ** 2 == pytest.approx(GOLD["F_CCZ"], rel=1e-14)


def test_xi_ccz_and_scaling():
    dec = decomp.gate_decomposition(("CCZ_SUM8", 0, 1, 2))
    assert sum(abs(c) for c, _ in dec) ** 2 == pytest.approx(GOLD["xi_CCZ"], rel=1e-14)
    t = decomp.gate_decomposition(("T", 0))
    xi_t = sum(abs(c) for c, _ in t) ** 2
    # a Toffoli costs 4 T gates: xi(T)^4 per Toffoli, xi(CCZ) per CCZ
    assert math.log2(xi_t ** 4) == pytest.approx(GOLD["T_scaling_log2_per_toffoli"], abs=1e-3)
    assert math.log2(GOLD["xi_CCZ"]) == pytest.approx(GOLD["CCZ_scaling_log2_per_toffoli"], abs=1e-2)
