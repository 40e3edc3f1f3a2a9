"""The trained selector against exhaustive timing (no GPU needed: the timing
table was measured on a GB300 by paper_1307_2100_gb300.selector, and the
host predictions use the same network as tc_plan's AUTO mapping).

Regret of a choice = t(choice) / t(best) - 1 over the held-out descriptors.
The target is a mean regret <= 0.10; the test also shows what the network
gains over the paper's class recipe, the method without it."""
import os

import numpy as np
import pytest

tc = pytest.importorskip("paper_1307_2100_gb300.tc")
from paper_1307_2100_gb300 import selector as sel  # noqa: E402

DATA = os.path.join(os.path.dirname(sel.__file__), "data")
WEIGHTS = os.path.join(DATA, "selector_gb300.bin")
TIMINGS = os.path.join(DATA, "selector_timings_gb300.npz")


@pytest.fixture(scope="module")
def result():
    if not (os.path.exists(WEIGHTS) and os.path.exists(TIMINGS)):
        pytest.skip("no trained selector")
    return sel.evaluate(TIMINGS, WEIGHTS, holdout=2000, use_gpu=False)


def test_selector_regret_target(result):
    assert result["n"] >= 1900
    assert result["network"]["mean"] <= 0.10
    assert result["network"]["median"] <= 0.05


def test_selector_gains_over_the_recipe(result):
    assert result["network"]["mean"] < 0.5 * result["recipe"]["mean"]
    assert result["total_time_ms"]["network"] < result["total_time_ms"]["recipe"]
    # no single fixed mapping does as well either
    for c in sel.CANDIDATES:
        assert result["network"]["mean"] < result["always_" + c]["mean_regret_where_feasible"]


def test_held_out_descriptors_were_not_trained_on():
    tr, te = sel.split(20000, 2000)
    assert len(set(tr) & set(te)) == 0 and len(te) == 2000
