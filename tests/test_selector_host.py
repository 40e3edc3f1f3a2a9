"""Host side of the learned selector (no GPU): the selector file round trip,
host predictions against an FP64 forward of the FP16 weights, and tc_plan's
AUTO mapping choosing the predicted-fastest candidate or falling back to the
paper's recipe."""
import numpy as np
import pytest

import tcsynth as ts
from oracle import mlp

tc = pytest.importorskip("paper_1307_2100_gb300.tc")
from paper_1307_2100_gb300 import selector as sel  # noqa: E402

F, H = tc.N_FEATURES, sel.HIDDEN
C = len(sel.CANDIDATES)


def _write(path, params, lo=None, hi=None, mean=None, scale=None, ym=0.0, ys=1.0):
    lo = np.full(F, -1e9, np.float32) if lo is None else lo
    hi = np.full(F, 1e9, np.float32) if hi is None else hi
    mean = np.zeros(F, np.float32) if mean is None else mean
    scale = np.ones(F, np.float32) if scale is None else scale
    sel.write_weights(path, F, H, C, sel.CAND_IDS, lo, hi, mean, scale, ym, ys, params)


def test_selector_file_round_trip_and_prediction(tmp_path):
    rng = np.random.default_rng(0)
    n = mlp.n_params(F, H, C)
    params = rng.normal(0, 0.1, n).astype(np.float32)
    mean = rng.normal(0, 0.2, F).astype(np.float32)
    scale = rng.uniform(0.5, 2, F).astype(np.float32)
    path = str(tmp_path / "sel.bin")
    _write(path, params, mean=mean, scale=scale, ym=3.0, ys=2.0)
    X = rng.uniform(0, 1, (17, F)).astype(np.float32)
    tc.tc_selector_load(path)
    try:
        pred, cand = tc.tc_selector_predict(X)
    finally:
        tc.tc_selector_unload()
    assert list(cand) == sel.CAND_IDS
    theta = params.astype(np.float16).astype(np.float64)
    y, _ = mlp.forward(theta, (X - mean) * scale, F, H, C)
    np.testing.assert_allclose(pred, y * 2.0 + 3.0, rtol=1e-4, atol=1e-4)


def test_malformed_selector_file_is_rejected(tmp_path):
    p = tmp_path / "bad.bin"
    p.write_bytes(b"TCSEL01\0" + b"\x01\x00")
    with pytest.raises(tc.TcError) as e:
        tc.tc_selector_load(str(p))
    assert e.value.status == 1
    with pytest.raises(tc.TcError) as e:
        tc.tc_selector_predict(np.zeros((1, F), np.float32))
    assert e.value.status == 9   # no selector loaded


def _plan_choice(p):
    h = tc.tc_plan((p.A.labels, p.A.extents, p.A.strides), (p.B.labels, p.B.extents, p.B.strides),
                   (p.C.labels, p.C.extents, p.C.strides), tc.TC_F32, tc.MATH["bf16x6"])
    try:
        info = tc.tc_plan_get_info(h)
        return tc.MAPPING_NAME[info.mapping], info.tile
    finally:
        tc.tc_plan_destroy(h)


def _plan_mapping(p):
    return _plan_choice(p)[0]


SPEC = {name: (m, t) for name, m, t in sel.CANDIDATE_SPECS}


@pytest.mark.parametrize("favoured", ["dot", "copy_gemm", "copy_gemm_gather", "gemv",
                                      "fused_gemm_gather"])
def test_auto_mapping_follows_the_selector(tmp_path, favoured):
    # a network whose output is its bias alone: the favoured candidate is fastest
    n = mlp.n_params(F, H, C)
    params = np.zeros(n, np.float32)
    b3 = np.full(C, 10.0, np.float32)
    b3[sel.CANDIDATES.index(favoured)] = 1.0
    params[-C:] = b3
    path = str(tmp_path / "sel.bin")
    _write(path, params)
    p3 = ts.fused_permute_48(n=6)           # Class 3.1
    p2 = ts.gemv_1024(a=6, b=5, i=7)        # Class 2
    assert _plan_choice(p3) == ("fused_gemm", 3)  # the recipe without a selector
    tc.tc_selector_load(path)
    try:
        m, t = SPEC[favoured]
        got = _plan_choice(p3)
        assert got[0] == m and (t < 0 or got[1] == t), got
        # COPY+GEMM cannot compute a Class 2 contraction: the first of the
        # equally predicted others (fused_gemm on packed operands) is used
        m2, t2 = (m, t) if m != "copy_gemm" else ("fused_gemm", 3)
        got2 = _plan_choice(p2)
        assert got2[0] == m2 and (t2 < 0 or got2[1] == t2), got2
    finally:
        tc.tc_selector_unload()
    assert _plan_choice(p3) == ("fused_gemm", 3)


def test_explicit_tile_overrides_the_selector(tmp_path):
    n = mlp.n_params(F, H, C)
    params = np.zeros(n, np.float32)
    b3 = np.full(C, 10.0, np.float32)
    b3[sel.CANDIDATES.index("fused_gemm_gather")] = 1.0
    params[-C:] = b3
    path = str(tmp_path / "sel.bin")
    _write(path, params)
    p = ts.fused_permute_48(n=6)
    tc.tc_selector_load(path)
    try:
        h = tc.tc_plan(_t(p.A), _t(p.B), _t(p.C), tc.TC_F32, tc.MATH["bf16x6"], 0, 3)
        try:
            info = tc.tc_plan_get_info(h)
            assert tc.MAPPING_NAME[info.mapping] == "fused_gemm" and info.tile == 3
        finally:
            tc.tc_plan_destroy(h)
    finally:
        tc.tc_selector_unload()


def _t(t):
    return (t.labels, t.extents, t.strides)


def test_auto_falls_back_to_recipe_outside_training_range(tmp_path):
    n = mlp.n_params(F, H, C)
    params = np.zeros(n, np.float32)
    params[-C:] = np.where(np.array(sel.CANDIDATES) == "dot", 1.0, 5.0)   # would pick dot
    lo = np.full(F, 10.0, np.float32)                      # every feature below range
    hi = np.full(F, 11.0, np.float32)
    path = str(tmp_path / "sel.bin")
    _write(path, params, lo=lo, hi=hi)
    tc.tc_selector_load(path)
    try:
        assert _plan_mapping(ts.fused_permute_48(n=6)) == "fused_gemm"
    finally:
        tc.tc_selector_unload()


def test_regret_and_feasibility_helpers():
    r = sel.regret_stats(np.array([1.0, 2.0, 3.0]), np.array([1.0, 1.0, 2.0]))
    assert r["mean"] == pytest.approx((0 + 1 + 0.5) / 3)
    ok = sel.feasible(np.array([1, 2, 31, 32]))
    assert ok[:2, sel.CANDIDATES.index("slice_gemm")].sum() == 0
    assert ok[2:].all()
