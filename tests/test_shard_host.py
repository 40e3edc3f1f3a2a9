"""Free-index sharding (tc_shard_free_index, paper_1307_2100_gb300.shard) on
the host: the shards' ranges partition C's largest free index in balanced
pieces, and the slabs, contracted one by one by the oracle at the shards'
buffer offsets, give the whole contraction bit for bit (each output's sum is
the same sum whichever slab holds it).  Two gloo ranks check the rank logic:
each contracts only its own slab (no data crosses ranks during the
contraction; the test gathers the slabs afterwards to compare)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import tcsynth as ts

tc = pytest.importorskip("paper_1307_2100_gb300.tc")
from paper_1307_2100_gb300 import shard as sh  # noqa: E402


def _descs(p):
    return [(t.labels, t.extents, t.strides) for t in (p.A, p.B, p.C)]


def contract_slab(p, n, r, cbuf):
    """Shard r of n of problem p contracted by the oracle into cbuf (C's buffer)."""
    s, (a, b, c) = sh.slab(*_descs(p), n, r)
    if s.end <= s.begin:
        return s
    oracle.contract_raw(a[0], a[1], a[2], np.asarray(p.A.data[s.offset_a:], np.float64),
                        b[0], b[1], b[2], np.asarray(p.B.data[s.offset_b:], np.float64),
                        c[0], c[1], c[2], cbuf[s.offset_c:], p.alpha, 0.0)
    return s


def problems():
    rng = np.random.Generator(np.random.PCG64(4242))
    out = [ts.direct_gemm_64(n=9), ts.fused_permute_48(n=7), ts.slice_gemm_48(),
           ts.problem("gemv", "aib", "i", "ab", dict(a=31, i=17, b=10), 3),
           ts.problem("dot", "ij", "ji", "", dict(i=7, j=9), 4),
           ts.problem("rowmajor_c", "ai", "ib", "ab", dict(a=20, i=6, b=33), 5, order_c=[1, 0])]
    out += [ts.random_problem(rng, max_order=4, max_ext=6) for _ in range(40)]
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_slabs_reassemble_the_contraction_bitwise(n):
    for p in problems():
        ref = oracle.contract_problem(p)
        cbuf = np.zeros(max(p.C.data.size, 1))
        spans = []
        for r in range(n):
            s = contract_slab(p, n, r, cbuf)
            spans.append((s.begin, s.end))
        np.testing.assert_array_equal(cbuf[: p.C.data.size], ref, err_msg=p.name)
        # the ranges partition the split index, in order, balanced
        if p.C.order:
            E = max(p.C.extents)
            assert spans[0][0] == 0 and spans[-1][1] == E
            assert all(spans[i][1] == spans[i + 1][0] for i in range(n - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def test_split_label_is_the_largest_free_index_larger_stride_on_ties():
    # C[a,b] with a = b = 40, column-major: ties go to b (stride 40)
    s = tc.tc_shard_free_index(([0, 2], [40, 7], None), ([2, 1], [7, 40], None),
                               ([0, 1], [40, 40], None), 4, 1)
    assert s.label == 1 and s.pos_c == 1 and (s.begin, s.end) == (10, 20)
    assert s.offset_c == 10 * 40 and s.offset_b == 10 * 7 and s.offset_a == 0
    # a larger extent wins over the stride
    s = tc.tc_shard_free_index(([0, 2], [50, 7], None), ([2, 1], [7, 40], None),
                               ([0, 1], [50, 40], None), 2, 1)
    assert s.label == 0 and (s.begin, s.end) == (25, 50) and s.offset_a == 25


def test_scalar_output_goes_to_shard_zero_and_errors():
    A, B, C = ([0, 1], [3, 4], None), ([1, 0], [4, 3], None), ([], [], None)
    s0 = tc.tc_shard_free_index(A, B, C, 3, 0)
    s2 = tc.tc_shard_free_index(A, B, C, 3, 2)
    assert s0.label == -1 and (s0.begin, s0.end) == (0, 1) and s2.end == 0
    for n, r in ((0, 0), (2, 2), (2, -1)):
        with pytest.raises(tc.TcError) as e:
            tc.tc_shard_free_index(A, B, C, n, r)
        assert e.value.status == 1
    with pytest.raises(tc.TcError) as e:           # extents of a label disagree
        tc.tc_shard_free_index(([0, 1], [3, 4], None), ([1, 2], [5, 6], None),
                               ([0, 2], [3, 6], None), 2, 0)
    assert e.value.status == 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = ts.direct_gemm_64(n=11)
        r, w = sh.rank_and_world()
        cbuf = np.zeros(p.C.data.size)
        s = contract_slab(p, w, r, cbuf)     # this rank's slab only
        part = torch.from_numpy(cbuf)
        dist.all_reduce(part)                 # gather the disjoint slabs to check them
        out[rank] = (r, w, int(s.begin), int(s.end),
                     bool(np.array_equal(part.numpy(), oracle.contract_problem(p))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_contract_their_own_slabs():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:4] == (0, 2, 0, 5) and res[1][:4] == (1, 2, 5, 11)
    assert res[0][4] and res[1][4]
