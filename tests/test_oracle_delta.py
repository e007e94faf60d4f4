"""Pins of the error-control measures (Sec. 2.6, Eq. 20-21) against values
worked out by hand from their definitions (tests/golden/delta_worked.json):
each case is built so that a plausible slip in the oracle -- a signed
difference, e_new in the norm, the upper median, a norm without the
median -- gives a different number."""
import json
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "delta_worked.json")
CASES = json.load(open(GOLDEN))["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_delta_cell_worked(orc, case):
    assert orc.delta(case["e_new"], case["e_old"], 0) == pytest.approx(case["delta_cell"], rel=1e-15)
    for wrong in case["mistakes_caught"].values():
        wrong = math.inf if wrong == "inf" else wrong
        assert wrong != pytest.approx(case["delta_cell"], rel=1e-6)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_delta_tot_worked(orc, case):
    num, den = case["delta_tot_exact"].split("/")
    assert case["delta_tot"] == pytest.approx(float(num) / float(den), rel=1e-15)
    assert orc.delta(case["e_new"], case["e_old"], 1) == pytest.approx(case["delta_tot"], rel=1e-15)


def test_delta_cell_ignores_cell_order(orc):
    """The measure is a max over cells with a median norm: permuting the
    cells (both arrays alike) leaves it unchanged."""
    c = CASES[0]
    perm = [5, 3, 0, 4, 1, 2]
    en = [c["e_new"][k] for k in perm]
    eo = [c["e_old"][k] for k in perm]
    assert orc.delta(en, eo, 0) == orc.delta(c["e_new"], c["e_old"], 0)
