"""Pins of the classification oracle against the paper's worked examples
(tests/golden/classification_cases.json, each case citing its section)."""
import json
import os

import numpy as np
import pytest

from oracle import classify as oc
import tcsynth as ts

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "classification_cases.json")))
NAMES = {}


def _id(name):
    return NAMES.setdefault(name, 1 + len(NAMES))


def _desc(names, n=4):
    labels = [_id(x) for x in names]
    ext = [n] * len(labels)
    return oc.Desc(labels, ext, ts.col_major(ext))


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_paper_case_class(case):
    A, B, C = _desc(case["A"]), _desc(case["B"]), _desc(case["C"])
    r = oc.classify(A, B, C)
    assert r.cls == case["cls"], case["cite"]
    if "recipe_A" in case:
        assert list(r.slice_a) == case["recipe_A"], case["cite"]


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_paper_case_slicings_lead_to_stated_kernel(case):
    A, B = _desc(case["A"]), _desc(case["B"])
    for s in case["slicings"]:
        assert oc.slicing_kernel(A, B, s["sA"], s["sB"]) == s["kernel"], s["cite"]


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_recipe_slicing_leads_to_the_class_kernel(case):
    A, B, C = _desc(case["A"]), _desc(case["B"]), _desc(case["C"])
    r = oc.classify(A, B, C)
    k = oc.slicing_kernel(A, B, r.slice_a, r.slice_b)
    want = {1: "DOT", 2: "GEMV", 31: "COPY+GEMM", 32: "GEMM"}[r.cls]
    assert k == want
    if r.cls == 32:
        req = oc.requirements(A, B, r.slice_a, r.slice_b)
        assert req["R1"] and req["R2"] and req["R3"] and req["consistent"]


def test_table1_by_rule():
    t = GOLD["table1"]
    A = _desc(t["A"])
    classes = {}
    for bl in t["B_variants"]:
        B = _desc(bl)
        free = [x for x in t["A"] if x not in bl] + [x for x in bl if x not in t["A"]]
        r = oc.classify(A, B, _desc(free))
        classes[" ".join(bl)] = r.cls
    for key, cls in t["highlighted"].items():
        assert classes[key] == cls
    c31 = sorted(k for k, v in classes.items() if v == 31)
    assert c31 == sorted(" ".join(b) for b in t["class31_by_rule"])
    assert sum(v == 32 for v in classes.values()) == 14
    assert len(classes) == 18


def test_fig3D2_recipe_is_one_of_the_two_gemm_slicings():
    case = [c for c in GOLD["cases"] if c["name"] == "fig3D2"][0]
    r = oc.classify(_desc(case["A"]), _desc(case["B"]), _desc(case["C"]))
    options = [(tuple(s["sA"]), tuple(s["sB"])) for s in case["slicings"]]
    assert (r.slice_a, r.slice_b) in options


def test_fig3D1_recipe_is_a_copy_gemm_slicing_of_the_paper():
    case = [c for c in GOLD["cases"] if c["name"] == "fig3D1"][0]
    r = oc.classify(_desc(case["A"]), _desc(case["B"]), _desc(case["C"]))
    options = [(tuple(s["sA"]), tuple(s["sB"])) for s in case["slicings"]
               if s["kernel"] == "COPY+GEMM"]
    assert (r.slice_a, r.slice_b) in options


def test_delta_counts_free_indices():
    # Sec. 3.2: Delta(t) = N(t) - p
    r = oc.classify(_desc(["i", "a", "j", "b"]), _desc(["j", "c", "i", "d"]),
                    _desc(["a", "b", "c", "d"]))
    assert (r.p, r.delta_a, r.delta_b) == (2, 2, 2)


def test_class3_has_gemm_for_relabelled_and_permuted_twins():
    """Random Class 3 descriptors: the class depends only on which index of
    each operand has stride 1 and whether it is contracted, so relabelling
    keeps the class, and storing the operands so that their stride-1 indices
    are free moves a Class 3.1 contraction into Class 3.2 (Sec. 3.3)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(200):
        p = ts.random_problem(rng, max_order=4, max_ext=4, min_ext=2, allow_outer=False)
        r = oc.classify(p.A, p.B, p.C)
        q_labels = {l: 500 - l for l in set(p.A.labels) | set(p.B.labels)}
        A2 = oc.Desc([q_labels[l] for l in p.A.labels], p.A.extents, p.A.strides)
        B2 = oc.Desc([q_labels[l] for l in p.B.labels], p.B.extents, p.B.strides)
        C2 = oc.Desc([q_labels[l] for l in p.C.labels], p.C.extents, p.C.strides)
        assert oc.classify(A2, B2, C2).cls == r.cls
        if r.cls in (31, 32) and r.free_a and r.free_b:
            def free_first(t, free):
                pos = t.labels.index(free[0])
                order = [pos] + [k for k in range(len(t.labels)) if k != pos]
                return oc.Desc(t.labels, t.extents, ts.storage_strides(t.extents, order))
            r2 = oc.classify(free_first(p.A, r.free_a), free_first(p.B, r.free_b), p.C)
            assert r2.cls == 32
