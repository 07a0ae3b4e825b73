"""The CPU oracle against what the paper and plain mathematics fix (no GPU)."""
import math

import pytest

import oracle
import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    """Object at a time (Sec. 2.2.4)."""
    pin(oracle.mdrq)


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_columnwise_pin(pin):
    """Dimension at a time (Sec. 3.2): held to the same pins on its own."""
    pin(oracle.mdrq_columnwise)


def test_closed_form_matches_paper_numbers():
    """The random-pair reading (interval from the smaller to the larger value per
    dimension) reproduces the selectivities printed in Sec. 7.4.1."""
    import json, os
    gold = json.load(open(os.path.join(pins.GOLDEN, "random_pair_selectivity.json")))
    n = gold["n"]
    m5 = pins.random_pair_closed_form(5, n)
    m10 = pins.random_pair_closed_form(10, n)
    m20 = pins.random_pair_closed_form(20, n)
    # printed to one significant figure / 2 significant figures
    assert round(100 * m5[0], 1) == gold["m5"]["mean_pct"]
    assert round(100 * m5[1], 1) == gold["m5"]["sd_pct"]
    assert round(100 * m10[0], 3) == gold["m10"]["mean_pct"]
    assert round(100 * m10[1], 2) == gold["m10"]["sd_pct"]
    assert math.isclose(100 * m20[0], gold["m_gt10"]["mean_pct"], rel_tol=1e-3)
