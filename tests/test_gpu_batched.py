"""GPU parity of the batched persistent launch (tc_contract_batched): every
item against the split-form oracle and the FP64 oracle, against the same
contraction run alone, and replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import magnitude, tc_bounds, within

pytestmark = pytest.mark.gpu


def _plans_and_buffers(items, form, mapping="auto"):
    import torch
    from paper_1307_2100_gb300 import Contraction
    dev = torch.device("cuda:0")
    plans, bufs = [], []
    for p in items:
        pl = Contraction((p.A.labels, p.A.extents, p.A.strides),
                         (p.B.labels, p.B.extents, p.B.strides),
                         (p.C.labels, p.C.extents, p.C.strides), "f32", form, mapping)
        plans.append(pl)
        A = torch.from_numpy(np.ascontiguousarray(p.A.data, np.float32)).to(dev)
        B = torch.from_numpy(np.ascontiguousarray(p.B.data, np.float32)).to(dev)
        C = torch.from_numpy(np.ascontiguousarray(p.C.data, np.float32)).to(dev)
        bufs.append((A, B, C))
    return plans, bufs


def _pointer_arrays(bufs, items):
    import torch
    dev = torch.device("cuda:0")
    ptr = lambda k: torch.tensor([b[k].data_ptr() for b in bufs], dtype=torch.int64, device=dev)
    alpha = torch.tensor([p.alpha for p in items], dtype=torch.float64, device=dev)
    beta = torch.tensor([p.beta for p in items], dtype=torch.float64, device=dev)
    return ptr(0), ptr(1), ptr(2), alpha, beta


def _run_batch(items, form):
    import torch
    from paper_1307_2100_gb300 import tc
    plans, bufs = _plans_and_buffers(items, form)
    batch = tc.tc_batch_plan([pl.handle for pl in plans])
    try:
        pa, pb, pc, al, be = _pointer_arrays(bufs, items)
        s = torch.cuda.current_stream().cuda_stream
        tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(),
                               al.data_ptr(), be.data_ptr(), s)
        torch.cuda.synchronize()
        assert tc.tc_device_status(s) == tc.TC_OK
        info = tc.tc_batch_get_info(batch)
    finally:
        tc.tc_batch_destroy(batch)
    return [b[2].cpu().numpy().astype(np.float64) for b in bufs], info


def _routes_to_tensor_cores(p, threshold=64):
    """The batch sends an item to the tensor cores when its GEMM view has M and
    N >= threshold (other items use exact FP32 products on the CUDA cores)."""
    from paper_1307_2100_gb300 import tc
    h = tc.tc_plan((p.A.labels, p.A.extents, p.A.strides), (p.B.labels, p.B.extents, p.B.strides),
                   (p.C.labels, p.C.extents, p.C.strides), tc.TC_F32, tc.MATH["bf16x6"])
    try:
        i = tc.tc_plan_get_info(h)
        return i.M >= threshold and i.N >= threshold
    finally:
        tc.tc_plan_destroy(h)


def small_items(n=48, seed=ts.BASE_SEED + 30):
    return ts.batching_items(n, seed=seed, max_elems=1 << 16, max_flops=float(1 << 26), lo=4,
                             hi=40)


def test_batched_routes_and_long_k_items():
    """Items of every class, including scalar results with long K, through both
    routes (tensor cores and the split-K CUDA-core kernels)."""
    from paper_1307_2100_gb300 import tc
    items = small_items(40, seed=ts.BASE_SEED + 34)
    items.append(ts.problem("dotlong", "ijk", "kji", "", dict(i=60, j=50, k=70), 35,
                            dtype=np.float32))
    items.append(ts.problem("gemvlong", "aib", "ib", "a", dict(a=300, i=200, b=90), 36,
                            dtype=np.float32))
    for p in items[-2:]:
        p.C.data = p.C.data.astype(np.float32)
    outs, info = _run_batch(items, "bf16x6")
    assert info.n_tc_items > 0 and info.n_simt_items > 0
    for p, got in zip(items, outs):
        acc, tot = tc_bounds(p, "bf16x6")
        ok, d = within(got, oracle.contract_problem(p), magnitude(p), p.C, tot)
        assert ok, (p.name, p.A.labels, p.B.labels, d)


def test_batched_degenerate_batches():
    """An empty batch runs nothing; one-item batches on either route alone (no
    second stream); an item with an empty output or an empty contracted range
    is refused when the batch is planned."""
    import torch
    from paper_1307_2100_gb300 import Contraction, tc
    empty = tc.tc_batch_plan([])
    try:
        assert tc.tc_batch_get_info(empty).n_items == 0
        tc.tc_contract_batched(empty, 0, 0, 0, 0, 0, torch.cuda.current_stream().cuda_stream)
    finally:
        tc.tc_batch_destroy(empty)
    f32 = np.float32
    gemv = ts.problem("one_gemv", "aib", "ib", "a", dict(a=300, i=70, b=9), 111, dtype=f32)
    gemm = ts.problem("one_gemm", "ai", "ib", "ab", dict(a=150, i=300, b=140), 112, dtype=f32)
    for p, route in ((gemv, 64), (gemm, 1)):
        tc.tc_batch_set_route(route)
        try:
            outs, info = _run_batch([p], "bf16x6")
        finally:
            tc.tc_batch_set_route(64)
        assert (info.n_tc_items, info.n_simt_items) == ((0, 1) if p is gemv else (1, 0))
        acc, tot = tc_bounds(p, "bf16x6")
        ok, d = within(outs[0], oracle.contract_problem(p), magnitude(p), p.C, tot)
        assert ok, (p.name, d)
    for ext in (dict(a=5, i=0, b=4), dict(a=0, i=3, b=4)):
        q = ts.problem("zero", "ai", "ib", "ab", ext, 113, dtype=f32)
        pl = Contraction((q.A.labels, q.A.extents, q.A.strides),
                         (q.B.labels, q.B.extents, q.B.strides),
                         (q.C.labels, q.C.extents, q.C.strides), "f32", "bf16x6", "auto")
        with pytest.raises(tc.TcError) as e:
            tc.tc_batch_plan([pl.handle])
        assert e.value.status == 5


def test_batched_split_k_tiles():
    """Tensor-core items whose tiles hold more K than half of one SM's share of
    the route's K blocks are split into K ranges: long-K items beside short
    ones, ragged tiles, alpha/beta, against the FP64 oracle at the BF16x6
    bound and against the split-form oracle."""
    from paper_1307_2100_gb300 import tc
    f32 = np.float32
    items = [
        ts.problem("s_long", "ai", "ib", "ab", dict(a=130, i=9000, b=70), 101, dtype=f32),
        ts.problem("s_multik", "aijb", "ijc", "abc", dict(a=9, i=61, j=67, b=15, c=129), 102,
                   dtype=f32),
        ts.problem("s_short", "ai", "ib", "ab", dict(a=200, i=40, b=150), 103, dtype=f32),
        ts.problem("s_ab", "ia", "ib", "ab", dict(a=100, i=5000, b=90), 104, dtype=f32),
    ]
    ab = items[-1]
    ab.C.data = np.linspace(-1, 1, ab.C.data.size).astype(f32)
    ab.alpha, ab.beta = 0.5, -2.0
    tc.tc_batch_set_route(1)
    try:
        outs, info = _run_batch(items, "bf16x6")
    finally:
        tc.tc_batch_set_route(64)
    assert info.n_simt_items == 0 and info.n_tc_split > 0
    for p, got in zip(items, outs):
        mag = magnitude(p)
        if p.beta != 0.0:
            mag = mag + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
        acc, tot = tc_bounds(p, "bf16x6")
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, tot)
        assert ok, (p.name, "fp64", d)
        ok, d = within(got, op.contract_form(p, "bf16x6"), mag, p.C, acc)
        assert ok, (p.name, "form", d)


def test_batched_cuda_core_tiles():
    """Skinny GEMMs (16 <= min(M, N) < the route threshold) take the 32 x 32
    tile kernel of the CUDA-core route: ragged tiles, K split into segments,
    several contracted labels, permuted storage orders, a batch label,
    alpha/beta.  Each block of 32 products is summed in FP32 (at most 32
    roundings of sum |a||b|), the block sums with Neumaier compensation, the
    result rounded once to FP32: 40 * 2^-24 of sum |a||b| covers it."""
    f32 = np.float32
    items = [
        ts.problem("t_longk", "ai", "ib", "ab", dict(a=38, i=20011, b=45), 91, dtype=f32),
        ts.problem("t_perm", "iajb", "jcid", "abcd", dict(i=7, a=20, j=9, b=3, c=17, d=2), 92,
                   dtype=f32),
        ts.problem("t_order", "kai", "ikb", "ab", dict(k=13, i=11, a=50, b=33), 93, dtype=f32,
                   order_a=[2, 0, 1], order_b=[1, 2, 0], order_c=[1, 0]),
        ts.problem("t_wide", "ai", "ib", "ab", dict(a=20, i=21, b=5000), 94, dtype=f32),
        ts.problem("t_batch", "aix", "ibx", "abx", dict(a=30, i=50, b=40, x=3), 95, dtype=f32),
        ts.problem("t_ab", "ia", "ib", "ab", dict(a=17, i=300, b=16), 96, dtype=f32),
    ]
    ab = items[-1]
    ab.C.data = np.linspace(-2, 2, ab.C.data.size).astype(f32)
    ab.alpha, ab.beta = -0.5, 1.5
    outs, info = _run_batch(items, "bf16x6")
    assert info.n_tc_items == 0 and info.n_simt_tiles > 0 and info.n_simt_work == 0
    for p, got in zip(items, outs):
        mag = magnitude(p)
        if p.beta != 0.0:  # outputs with beta = 0 start as NaN: C must not be read
            mag = mag + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, 40 * 2.0 ** -24)
        assert ok, (p.name, d)


@pytest.mark.parametrize("form", ["bf16x3", "bf16x6"])
def test_batched_items_against_oracles(form):
    items = small_items()
    outs, info = _run_batch(items, form)
    assert info.n_items == len(items)
    for p, got in zip(items, outs):
        mag = magnitude(p)
        acc, tot = tc_bounds(p, form)
        if _routes_to_tensor_cores(p):   # the split-form products are what it computes
            ok, d = within(got, op.contract_form(p, form), mag, p.C, acc)
            assert ok, (p.A.labels, p.B.labels, "method", d)
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, tot)
        assert ok, (p.A.labels, p.B.labels, "fp64", d)


def test_batched_alpha_beta():
    items = small_items(16, seed=ts.BASE_SEED + 31)
    rng = np.random.default_rng(5)
    for p in items:
        p.alpha = float(rng.uniform(-2, 2))
        p.beta = float(rng.uniform(-1, 1))
        p.C.data = rng.uniform(-1, 1, p.C.data.size).astype(np.float32)
    outs, _ = _run_batch(items, "bf16x6")
    for p, got in zip(items, outs):
        acc, _ = tc_bounds(p, "bf16x6")
        assert within(got, op.contract_form(p, "bf16x6"), magnitude(p), p.C, acc)[0]


def test_batched_graph_capture_and_replay():
    import torch
    from paper_1307_2100_gb300 import tc
    items = small_items(24, seed=ts.BASE_SEED + 32)
    plans, bufs = _plans_and_buffers(items, "bf16x6")
    batch = tc.tc_batch_plan([pl.handle for pl in plans])
    try:
        pa, pb, pc, al, be = _pointer_arrays(bufs, items)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(),
                                   al.data_ptr(), be.data_ptr(), s.cuda_stream)
        for rep in range(2):
            rng = np.random.default_rng(100 + rep)
            for p, (A, B, C) in zip(items, bufs):
                p.A.data = rng.uniform(-1, 1, p.A.data.size).astype(np.float32)
                p.B.data = rng.uniform(-1, 1, p.B.data.size).astype(np.float32)
                A.copy_(torch.from_numpy(p.A.data))
                B.copy_(torch.from_numpy(p.B.data))
                C.fill_(float("nan"))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            for p, (A, B, C) in zip(items, bufs):
                got = C.cpu().numpy().astype(np.float64)
                acc, _ = tc_bounds(p, "bf16x6")
                assert within(got, op.contract_form(p, "bf16x6"), magnitude(p), p.C, acc)[0]
    finally:
        tc.tc_batch_destroy(batch)


def test_batched_equals_single_launches_bitwise():
    """With every item routed to the tensor cores, the batched launch runs the
    same packed tiles with the same chunking as a lone tc_contract of a
    tensor-core plan on packed operands (tile 3), so those results agree bit
    for bit."""
    from gpu_util import run
    from paper_1307_2100_gb300 import tc
    items = small_items(20, seed=ts.BASE_SEED + 33)
    tc.tc_batch_set_route(1)
    try:
        outs, info = _run_batch(items, "bf16x6")
    finally:
        tc.tc_batch_set_route(64)
    assert info.n_simt_items == 0
    checked = 0
    for p, got in zip(items, outs):
        from paper_1307_2100_gb300 import Contraction
        plan = Contraction((p.A.labels, p.A.extents, p.A.strides),
                           (p.B.labels, p.B.extents, p.B.strides),
                           (p.C.labels, p.C.extents, p.C.strides), "f32", "bf16x6", "auto")
        if plan.info.as_dict()["kernel_name"] != "gemm_tc" or plan.info.batch != 1:
            continue
        single = run(p, "bf16x6", "auto", tile=3)
        np.testing.assert_array_equal(got, single)
        checked += 1
    assert checked >= 5


def test_batching_workload_every_item_against_oracle():
    """The bench's 512-item batching workload (BF16x3, the tensor-core and
    CUDA-core routes), every item against the FP64 oracle at the form's bound,
    and the tensor-core items against the split-form oracle."""
    items = ts.batching_items(512)
    outs, info = _run_batch(items, "bf16x3")
    assert info.n_tc_items > 50 and info.n_simt_items > 50
    bad = []
    for j, (p, got) in enumerate(zip(items, outs)):
        mag = magnitude(p)
        acc, tot = tc_bounds(p, "bf16x3")
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, tot)
        if not ok:
            bad.append((j, d))
    assert not bad, bad[:10]


def test_autotuned_routes():
    """The route and shape autotuner over the 512-item batching workload: the
    tuned batch is no slower than the threshold rule it starts from, every
    item takes one of the three shapes, and the tuned batch is within every
    item's bound of the FP64 oracle (routes change the arithmetic: BF16x3 or
    FP32)."""
    import torch
    from paper_1307_2100_gb300 import autotune, tc
    items = ts.batching_items(512)
    plans, bufs = _plans_and_buffers(items, "bf16x3")
    pa, pb, pc, al, be = _pointer_arrays(bufs, items)
    s = torch.cuda.Stream()
    routes, rep = autotune.tune_routes([pl.handle for pl in plans], (pa, pb, pc, al, be), s,
                                       reps=3)
    assert set(np.unique(routes)) <= {1, 2, 3}
    assert rep["tuned_ms"] <= rep["default_ms"]
    batch = tc.tc_batch_plan_routes([pl.handle for pl in plans], routes)
    try:
        for _, _, C in bufs:
            C.fill_(float("nan"))
        tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(), al.data_ptr(),
                               be.data_ptr(), s.cuda_stream)
        torch.cuda.synchronize()
    finally:
        tc.tc_batch_destroy(batch)
    for p, (_, _, C) in zip(items, bufs):
        got = C.cpu().numpy().astype(np.float64)[: p.C.data.size]
        _, tot = tc_bounds(p, "bf16x3")
        ok, d = within(got, oracle.contract_problem(p), magnitude(p), p.C, tot)
        assert ok, (p.name, d)


@pytest.mark.parametrize("shape", [2, 3])
def test_cuda_core_shapes_forced_on_every_item(shape):
    """Routes 2 (32 x 32 tiles) and 3 (a thread or warp per output) forced on
    every item, whatever its GEMM view: each within the CUDA-core route's FP32
    bound (40 * 2^-24 of sum |a||b|) of the FP64 oracle."""
    import torch
    from paper_1307_2100_gb300 import tc
    items = small_items()
    plans, bufs = _plans_and_buffers(items, "bf16x6")
    batch = tc.tc_batch_plan_routes([pl.handle for pl in plans], [shape] * len(items))
    try:
        pa, pb, pc, al, be = _pointer_arrays(bufs, items)
        for _, _, C in bufs:
            C.fill_(float("nan"))
        s = torch.cuda.current_stream().cuda_stream
        tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(), al.data_ptr(),
                               be.data_ptr(), s)
        torch.cuda.synchronize()
        info = tc.tc_batch_get_info(batch)
    finally:
        tc.tc_batch_destroy(batch)
    assert info.n_tc_items == 0
    assert (info.n_simt_work == 0) if shape == 2 else (info.n_simt_tiles == 0)
    for p, (_, _, C) in zip(items, bufs):
        got = C.cpu().numpy().astype(np.float64)[: p.C.data.size]
        mag = magnitude(p)
        if p.beta != 0.0:
            mag = mag + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, 40 * 2.0 ** -24)
        assert ok, (p.name, shape, d)

