"""The trained selectors against exhaustive timing (no GPU needed: the timing
tables were measured on a GB300 by paper_1307_2100_gb300.selector, and the
host predictions use the same networks as tc_plan's AUTO mapping).

Two selectors: FP32 storage with the BF16x6 form, and FP64 (whose candidates
include the CUDA-core GEMM's tile shapes).  Regret of a choice = t(choice) /
t(best) - 1 over the held-out descriptors.  The target is a mean regret
<= 0.10; the tests also show what each network gains over the paper's class
recipe, the method without it."""
import os

import numpy as np
import pytest

tc = pytest.importorskip("paper_1307_2100_gb300.tc")
from paper_1307_2100_gb300 import selector as sel  # noqa: E402

DATA = os.path.join(os.path.dirname(sel.__file__), "data")
FILES = {"bf16x6": ("selector_gb300.bin", "selector_timings_gb300.npz"),
         "fp64": ("selector_gb300_fp64.bin", "selector_timings_gb300_fp64.npz")}
_cache = {}


def result(kind):
    if kind not in _cache:
        w, t = (os.path.join(DATA, f) for f in FILES[kind])
        if not (os.path.exists(w) and os.path.exists(t)):
            pytest.skip("no trained selector")
        _cache[kind] = sel.evaluate(t, w, holdout=2000, use_gpu=False)
    return _cache[kind]


@pytest.mark.parametrize("kind", sorted(FILES))
def test_selector_regret_target(kind):
    r = result(kind)
    assert r["kind"] == kind and r["n"] >= 1900
    assert r["network"]["mean"] <= 0.10
    assert r["network"]["median"] <= 0.05


@pytest.mark.parametrize("kind", sorted(FILES))
def test_selector_gains_over_the_recipe(kind):
    r = result(kind)
    assert r["network"]["mean"] < 0.5 * r["recipe"]["mean"]
    assert r["total_time_ms"]["network"] < r["total_time_ms"]["recipe"]
    # no single fixed mapping does as well either
    for c, _m, _t in sel.specs(kind):
        assert r["network"]["mean"] < r["always_" + c]["mean_regret_where_feasible"]


def test_held_out_descriptors_were_not_trained_on():
    tr, te = sel.split(20000, 2000)
    assert len(set(tr) & set(te)) == 0 and len(te) == 2000


def test_fp64_descriptors_are_the_bounded_prefix():
    """The fp64 kind's descriptors are the selector workload's with at most
    2^34 flops, in order, whatever n asks for."""
    import tcsynth as ts
    d40 = sel.descriptors("fp64", 40, 7)
    d25 = sel.descriptors("fp64", 25, 7)
    assert [str(x) for x in d25] == [str(x) for x in d40[:25]]
    assert all(sel._flops(x) <= 2.0 ** 34 for x in d40)
    allx = [x for x in ts.selector_descriptors(60, seed=7) if sel._flops(x) <= 2.0 ** 34]
    assert [str(x) for x in d40] == [str(x) for x in allx[:40]]
