"""Host-side logic of the serving loop and the memory-footprint query (no GPU)."""
import pytest

import paper_2405_13973_gb300 as pt
from paper_2405_13973_gb300.serving import first_fit


def test_first_fit_admits_in_arrival_order_past_a_job_that_does_not_fit():
    waiting = [(50, "a"), (80, "b"), (30, "c"), (10, "d")]
    assert first_fit(waiting, used=0, budget=100, slots=10) == [0, 2, 3]
    assert first_fit(waiting, used=60, budget=100, slots=10) == [2, 3]
    assert first_fit(waiting, used=0, budget=100, slots=1) == [0]
    assert first_fit(waiting, used=0, budget=5, slots=10) == []


def test_footprint_grows_with_ions_and_shares_operators():
    a, oa = pt.plan_footprint(1000, 12, precision="bf16x3")
    b, ob = pt.plan_footprint(20000, 12, precision="bf16x3")
    c, oc = pt.plan_footprint(20000, 12, precision="fp64")
    assert 0 < a < b and oa == ob                 # operators do not depend on N
    assert oc != ob and c > 0
    # tensor-core modes support p <= 15
    with pytest.raises(pt.PenningError):
        pt.plan_footprint(1000, 16, precision="bf16x3")
    assert pt.plan_footprint(1000, 16, precision="fp64")[0] > 0
